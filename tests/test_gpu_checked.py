"""Failure detection without a GPU fault.

  * The checked build (libstereo_checked.so, in-kernel index checks that
    record a failure in a device error word and skip the access) runs the
    whole path, the stage entry points and the batched form on odd sizes,
    small and large windows and disparity ranges, and the whole path at the
    benchmark sizes: the error word stays 0 and every output equals the
    normal build's bit for bit.
  * Its self-test launches one check that cannot pass (its store is
    skipped): the error word reports the site, and reading it clears it.
  * Allocation failures injected at every device allocation of
    stereo_create (batched handles have seven): the call returns
    STEREO_ERR_OOM and the library holds no more allocations than before.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    st.lib()
    return torch.device("cuda:0")


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


KEYS = ("disp_wta", "disp_sub", "disp_lr", "disp_post", "valid", "disp_final")


def _outs(dev, H, W):
    return dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                disp_sub=torch.empty((H, W), dtype=torch.float32, device=dev),
                disp_lr=torch.empty((H, W), dtype=torch.int16, device=dev),
                disp_post=torch.empty((H, W), dtype=torch.int16, device=dev),
                valid=torch.empty((H, W), dtype=torch.uint8, device=dev),
                disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))


def _whole_path(dev, L, R, d_min, D, r, cdt, smooth):
    H, W = L.shape[:2]
    h = st.stereo_create(st.stereo_default_params(max_width=W, max_height=H, d_min=d_min, num_disp=D,
                                                  win_radius=r, cost_dtype=cdt, smooth_radius=smooth))
    o = _outs(dev, H, W)
    st.stereo_match(h, T(L, dev), T(R, dev), **o)
    # stage entry points on the whole path's maps
    lr = torch.empty_like(o["disp_lr"])
    post = torch.empty_like(o["disp_post"])
    st.stereo_stage_outlier(h, o["disp_lr"], 10, 2.5, lr)
    st.stereo_stage_postprocess(h, o["disp_lr"], post)
    torch.cuda.synchronize()
    err = st.stereo_get_device_error(h)
    h.close()
    res = {k: v.cpu().numpy() for k, v in o.items()}
    res["stage_outlier"] = lr.cpu().numpy()
    res["stage_post"] = post.cpu().numpy()
    return err, res


CASES = [((37, 23), 0, 5, 1, st.COST_F32, 2),        # odd sizes, tiny range and window
         ((101, 67), -3, 40, 7, st.COST_F16, 15),     # largest window, K = 2, negative first disparity
         ((173, 91), 0, 100, 5, st.COST_BF16, 15),    # K = 4 with lanes beyond the range
         ((230, 60), 2, 150, 4, st.COST_NONE, 3)]     # two chunks (128 at K = 4, 22 at K = 2), no volume


@pytest.mark.parametrize("size,d_min,D,r,cdt,smooth", CASES)
def test_checked_build_whole_path(dev, size, d_min, D, r, cdt, smooth):
    W, H = size
    Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(8, W), W, H, max(1.0, d_min + 1.0), d_min + 0.7 * D)
    err0, ref = _whole_path(dev, Lrgb, Rrgb, d_min, D, r, cdt, smooth)
    assert err0 == 0
    with st.checked_library():
        err, got = _whole_path(dev, Lrgb, Rrgb, d_min, D, r, cdt, smooth)
    assert err == 0, hex(err)
    for k in ref:
        assert np.array_equal(np.nan_to_num(ref[k], nan=-7), np.nan_to_num(got[k], nan=-7)), k


@pytest.mark.parametrize("size,d_min,D,r,cdt,smooth", [((960, 540), 0, 128, 5, st.COST_F32, 15),
                                                        ((960, 540), 0, 192, 7, st.COST_F16, 15)])
def test_checked_build_whole_path_full_size(dev, size, d_min, D, r, cdt, smooth):
    """The benchmark sizes (960x540 at D = 128, FP32, and D = 192, 15x15,
    FP16): no failed index check, the normal build's outputs bit for bit."""
    W, H = size
    Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(1), W, H, 10.0, 0.85 * D)
    err0, ref = _whole_path(dev, Lrgb, Rrgb, d_min, D, r, cdt, smooth)
    assert err0 == 0
    with st.checked_library():
        err, got = _whole_path(dev, Lrgb, Rrgb, d_min, D, r, cdt, smooth)
    assert err == 0, hex(err)
    for k in ref:
        assert np.array_equal(np.nan_to_num(ref[k], nan=-7), np.nan_to_num(got[k], nan=-7)), k


@pytest.mark.parametrize("size,d_min,D,r,cdt,smooth,sampling", [
    ((101, 45), 6, 80, 5, st.COST_F32, 5, st.SAMPLE_FULL),        # first disparity > 0, FP32 volume
    ((505, 29), 5, 225, 7, st.COST_F32, 5, st.SAMPLE_CHESSBOARD),  # short image: tile rows below it
    ((662, 224), 6, 246, 7, st.COST_F32, 5, st.SAMPLE_FULL),
    ((130, 50), 3, 70, 3, st.COST_F16, 15, st.SAMPLE_FULL)])
def test_checked_build_positive_first_disparity(dev, size, d_min, D, r, cdt, smooth, sampling):
    """A positive first disparity with a stored volume: the o-update's pixels
    without candidates (invalid ones, and the tile rows below a short image)
    fetch no candidate run (they once read from before their cost slice or
    past the volume's end)."""
    W, H = size
    Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(8, 1000 + W), W, H, d_min + 1.0, d_min + 0.8 * D)

    def run():
        h = st.stereo_create(st.stereo_default_params(max_width=W, max_height=H, d_min=d_min, num_disp=D,
                                                      win_radius=r, cost_dtype=cdt, smooth_radius=smooth,
                                                      sampling=sampling))
        o = _outs(dev, H, W)
        st.stereo_match(h, T(Lrgb, dev), T(Rrgb, dev), **o)
        torch.cuda.synchronize()
        err = st.stereo_get_device_error(h)
        h.close()
        return err, {k: v.cpu().numpy() for k, v in o.items()}

    err0, ref = run()
    with st.checked_library():
        err, got = run()
    assert err0 == 0 and err == 0, hex(err)
    for k in ref:
        assert np.array_equal(np.nan_to_num(ref[k], nan=-7), np.nan_to_num(got[k], nan=-7)), k


def test_maximum_size_pair(dev):
    """The largest range and window at 3840x2160 (D = 256, 15x15, FP16
    volume, 4.2 GB): no failed index check in the checked build, its outputs
    equal to the normal build's, and the winners of a 12-row strip equal to
    the oracle's (near-ties exempt)."""
    from parity import NEAR_TIE, int_map_mismatch, oracle_match_rows
    import oracle
    W, H, D, r = 3840, 2160, 256, 7
    Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(12, W), W, H, 10.0, 0.85 * D)

    def run():
        h = st.stereo_create(st.stereo_default_params(max_width=W, max_height=H, num_disp=D, win_radius=r,
                                                      cost_dtype=st.COST_F16))
        o = dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                 disp_post=torch.empty((H, W), dtype=torch.int16, device=dev),
                 disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))
        s = torch.cuda.Stream()
        st.stereo_match(h, T(Lrgb, dev), T(Rrgb, dev), **o, stream=s)
        s.synchronize()
        err = st.stereo_get_device_error(h)
        h.close()
        return err, {k: v.cpu().numpy() for k, v in o.items()}

    with st.checked_library():
        err, got = run()
    assert err == 0, hex(err)
    err0, ref = run()
    assert err0 == 0
    for k in ref:
        assert np.array_equal(np.nan_to_num(ref[k], nan=-7), np.nan_to_num(got[k], nan=-7)), k
    y0, y1 = 1400, 1412
    m = oracle_match_rows(oracle.gray(Lrgb), oracle.gray(Rrgb), 0, D, r, 0, y0, y1)
    bad = int_map_mismatch(ref["disp_wta"][y0:y1], m["dL"], m["gapL"] < NEAR_TIE)
    assert len(bad) == 0


def test_checked_build_batched(dev):
    """A batch of odd-size pairs in both stage modes: no failed check, the
    normal build's outputs."""
    shapes = [(45, 77, 0, 33, 3), (60, 130, -2, 64, 6), (31, 200, 0, 150, 5)]

    def run():
        pairs = []
        for i, (H, W, d_min, D, r) in enumerate(shapes):
            Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(8, 100 + i), W, H, max(1.0, d_min + 1.0),
                                               d_min + 0.7 * D)
            pairs.append(dict(left=T(Lrgb, dev), right=T(Rrgb, dev), d_min=d_min, num_disp=D, win_radius=r,
                              disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                              disp_post=torch.empty((H, W), dtype=torch.int16, device=dev),
                              disp_final=torch.empty((H, W), dtype=torch.float32, device=dev)))
        h = st.stereo_create(st.stereo_default_params(max_width=200, max_height=60, num_disp=150,
                                                      cost_dtype=st.COST_F16), max_batch=len(pairs))
        out = []
        for mode in (0, 1):
            st.stereo_set_batch_stages(h, mode)
            st.stereo_match_batched(h, pairs, use_graph=False)
            torch.cuda.synchronize()
            out.append([{k: p[k].cpu().numpy() for k in ("disp_wta", "disp_post", "disp_final")} for p in pairs])
        err = st.stereo_get_device_error(h)
        h.close()
        return err, out

    err0, ref = run()
    with st.checked_library():
        err, got = run()
    assert err0 == 0 and err == 0, hex(err)
    for mode in (0, 1):
        for a, b in zip(ref[mode], got[mode]):
            for k in a:
                assert np.array_equal(np.nan_to_num(a[k], nan=-7), np.nan_to_num(b[k], nan=-7)), (mode, k)


def test_checked_build_selftest_reports_and_clears(dev):
    with st.checked_library() as LC:
        h = st.stereo_create(st.stereo_default_params(max_width=32, max_height=16, num_disp=8))
        assert st.stereo_get_device_error(h) == 0
        assert LC.stereo_debug_check_selftest(None) == 0
        torch.cuda.synchronize()
        assert st.stereo_get_device_error(h) == 0x1000 | 0xfff
        assert st.stereo_get_device_error(h) == 0          # read and cleared
        h.close()


@pytest.mark.parametrize("max_batch,allocs", [(1, 2), (3, 7)])
def test_injected_allocation_failures_leave_nothing_behind(dev, max_batch, allocs):
    L = st.lib()
    p = st.stereo_default_params(max_width=96, max_height=64, num_disp=32)
    live0 = st.stereo_debug_live_allocations()
    for n in range(allocs):
        st.stereo_debug_fail_alloc(n)
        h = C.c_void_p()
        assert L.stereo_create(C.byref(p), max_batch, C.byref(h)) == 3, n      # STEREO_ERR_OOM
        assert st.stereo_debug_live_allocations() == live0, n
    st.stereo_debug_fail_alloc(allocs)                 # beyond the last allocation: no failure
    h = st.stereo_create(p, max_batch)
    assert st.stereo_debug_live_allocations() == live0 + allocs
    st.stereo_debug_fail_alloc(-1)
    h.close()
    assert st.stereo_debug_live_allocations() == live0
