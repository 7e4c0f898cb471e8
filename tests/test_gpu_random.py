"""Seeded random configurations (sizes, first disparity, range, window,
sampling, cost format, method parameters), beyond the fixed shapes of the
other tests.

  * test_random_parity: the cost/WTA stage against the oracle (both winner
    maps bit-exact outside near-ties, sub-pixel within 0.01 px, the FP32
    volume within 1e-6 of the FP64 ZNCC) and the oracle's left-right check
    and post-processing applied to the GPU's winners against the GPU's whole
    path, bit for bit.
  * test_random_checked: the whole path with random method parameters in the
    checked build (in-kernel index checks): no failed check, and the normal
    build's outputs bit for bit.  The checked build runs first, so a failed
    check is reported before the normal build makes the access.
  * test_random_subpixel_across_cost_types: the cost/WTA stage for the four
    cost formats (three ways of fitting the sub-pixel parabola), winners and
    sub-pixel disparities bit-identical, checked and normal builds.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import NEAR_TIE, SUB_TOL, int_map_mismatch

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


def _images(rng, W, H, d_min, D):
    if rng.integers(0, 3) == 0:
        return (rng.integers(0, 256, (H, W), dtype=np.uint8), rng.integers(0, 256, (H, W), dtype=np.uint8))
    Lrgb, Rrgb, _ = synth.tissue_pair(int(rng.integers(1 << 30)), W, H, max(1.0, d_min + 1.0), d_min + 0.8 * D)
    return oracle.gray(Lrgb), oracle.gray(Rrgb)


@pytest.mark.parametrize("case", range(24))
def test_random_parity(dev, case):
    rng = np.random.default_rng(synth.seed_for(9, case))
    W, H = int(rng.integers(20, 160)), int(rng.integers(16, 90))
    r, D, d_min = int(rng.integers(1, 8)), int(rng.integers(1, 200)), int(rng.integers(-30, 31))
    sampling = int(rng.choice([st.SAMPLE_FULL, st.SAMPLE_FULL, st.SAMPLE_CHESSBOARD]))
    L, R = _images(rng, W, H, d_min, D)
    p = st.stereo_default_params(max_width=W, max_height=H, d_min=d_min, num_disp=D, win_radius=r,
                                 cost_dtype=st.COST_F32, sampling=sampling, smooth_radius=5)
    h = st.stereo_create(p)
    dl = torch.empty((H, W), dtype=torch.int16, device=dev)
    dr = torch.empty_like(dl)
    sub = torch.empty((H, W), dtype=torch.float32, device=dev)
    cost = torch.zeros((H, W, st.cost_stride(D)), dtype=torch.float32, device=dev)
    st.stereo_stage_match(h, T(L, dev), T(R, dev), d_min, D, r, sampling, st.COST_F32, dl, dr, sub, cost)
    o = {k: torch.empty((H, W), dtype=torch.int16, device=dev) for k in ("disp_wta", "disp_lr", "disp_post")}
    st.stereo_match(h, T(L, dev), T(R, dev), **o)
    torch.cuda.synchronize()
    assert st.stereo_get_device_error(h) == 0
    h.close()
    gL, gR, gs = dl.cpu().numpy(), dr.cpu().numpy(), sub.cpu().numpy()
    m = oracle.match(L, R, d_min, D, r, sampling)
    assert len(int_map_mismatch(gL, m["dL"], m["gapL"] < NEAR_TIE)) == 0
    assert len(int_map_mismatch(gR, m["dR"], m["gapR"] < NEAR_TIE)) == 0
    same = (gL == m["dL"]) & (m["dL"] != oracle.INVALID)
    if same.any():
        assert np.max(np.abs(gs[same] - m["sub"][same])) <= SUB_TOL
    cv = oracle.cost_volume(L, R, d_min, D, r, sampling)
    gc = cost.cpu().numpy()[:, :, :D]
    assert np.array_equal(np.isnan(gc), np.isnan(cv))
    ok = ~np.isnan(cv)
    if ok.any():
        assert np.max(np.abs(gc[ok] - cv[ok])) <= 1e-6
    lr = oracle.lr_check(gL, gR, 1)
    assert np.array_equal(o["disp_wta"].cpu().numpy(), gL)
    assert np.array_equal(o["disp_lr"].cpu().numpy(), lr)
    assert np.array_equal(o["disp_post"].cpu().numpy(), oracle.postprocess(lr, oracle.Params()))


def _whole(dev, L, R, prm, W, H):
    h = st.stereo_create(prm)
    o = dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
             disp_sub=torch.empty((H, W), dtype=torch.float32, device=dev),
             disp_lr=torch.empty((H, W), dtype=torch.int16, device=dev),
             disp_post=torch.empty((H, W), dtype=torch.int16, device=dev),
             valid=torch.empty((H, W), dtype=torch.uint8, device=dev),
             disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))
    s = torch.cuda.Stream()
    st.stereo_match(h, T(L, dev), T(R, dev), **o, stream=s)
    s.synchronize()
    err = st.stereo_get_device_error(h)
    h.close()
    return err, {k: v.cpu().numpy() for k, v in o.items()}


@pytest.mark.parametrize("case", range(24))
def test_random_checked(dev, case):
    rng = np.random.default_rng(synth.seed_for(10, case))
    W, H = int(rng.integers(20, 500)), int(rng.integers(16, 300))
    r, D, d_min = int(rng.integers(1, 8)), int(rng.integers(1, 257)), int(rng.integers(-40, 41))
    cdt = int(rng.choice([st.COST_NONE, st.COST_F32, st.COST_F16, st.COST_BF16]))
    sampling = int(rng.choice([st.SAMPLE_FULL, st.SAMPLE_FULL, st.SAMPLE_CHESSBOARD]))
    extra = dict(lr_thresh=int(rng.integers(0, 4)), outlier_rounds=int(rng.integers(0, 4)),
                 r0=int(rng.integers(0, 40)), dr=int(rng.integers(0, 30)),
                 outlier_thresh=float(rng.choice([0.5, 2.5, 10.0])), fill_radial_r=int(rng.integers(1, 90)),
                 fill_radial_min_dirs=int(rng.integers(1, 9)), fill_disc_r=int(rng.integers(1, 57)),
                 fill_disc_min_count=int(rng.choice([-1, 1, 50])), smooth_radius=int(rng.choice([0, 2, 5, 15, 40])),
                 smooth_iters=int(rng.integers(0, 7)), refine_search=int(rng.integers(0, 9)))
    L, R = _images(rng, W, H, d_min, D)
    prm = st.stereo_default_params(max_width=W, max_height=H, d_min=d_min, num_disp=D, win_radius=r,
                                   cost_dtype=cdt, sampling=sampling, **extra)
    with st.checked_library():
        err, got = _whole(dev, L, R, prm, W, H)
    assert err == 0, hex(err)
    err0, ref = _whole(dev, L, R, prm, W, H)
    assert err0 == 0
    for k in ref:
        assert np.array_equal(np.nan_to_num(ref[k], nan=-7), np.nan_to_num(got[k], nan=-7)), k


def _stage_match(dev, L, R, d_min, D, r, cdt):
    H, W = L.shape
    p = st.stereo_default_params(max_width=W, max_height=H, num_disp=D, d_min=d_min, win_radius=r,
                                 cost_dtype=cdt)
    h = st.stereo_create(p)
    dl = torch.empty((H, W), dtype=torch.int16, device=dev)
    dr = torch.empty_like(dl)
    sub = torch.empty((H, W), dtype=torch.float32, device=dev)
    cost = None
    if cdt != st.COST_NONE:
        tdt = {st.COST_F32: torch.float32, st.COST_F16: torch.float16, st.COST_BF16: torch.bfloat16}[cdt]
        cost = torch.zeros((H, W, st.cost_stride(D)), dtype=tdt, device=dev)
    st.stereo_stage_match(h, T(L, dev), T(R, dev), d_min, D, r, st.SAMPLE_FULL, cdt, dl, dr, sub, cost)
    torch.cuda.synchronize()
    err = st.stereo_get_device_error(h)
    h.close()
    return err, dl.cpu().numpy(), dr.cpu().numpy(), sub.cpu().numpy()


@pytest.mark.parametrize("case", range(16))
def test_random_subpixel_across_cost_types(dev, case):
    """Random sizes, windows and ranges up to 256 disparities (one chunk, a
    split range, two chunks), first disparities down to -130 so that winners
    fall on both sides of the chunk edge: the sub-pixel parabola fitted by
    the finalize kernel from an FP32 volume, by the cost kernel itself (one
    chunk), or from the per-chunk winner costs (several chunks) gives the
    same winners and bit-identical sub-pixel disparities for the four cost
    types, in the checked build (no failed index check) and the normal one."""
    rng = np.random.default_rng(synth.seed_for(12, case))
    W, H = int(rng.integers(20, 400)), int(rng.integers(16, 160))
    r, D, d_min = int(rng.integers(1, 8)), int(rng.integers(1, 257)), int(rng.integers(-130, 40))
    L, R = _images(rng, W, H, d_min, D)
    ref = None
    for checked in (True, False):
        for cdt in (st.COST_F32, st.COST_F16, st.COST_BF16, st.COST_NONE):
            if checked:
                with st.checked_library():
                    err, dl, dr, sub = _stage_match(dev, L, R, d_min, D, r, cdt)
            else:
                err, dl, dr, sub = _stage_match(dev, L, R, d_min, D, r, cdt)
            assert err == 0, (hex(err), cdt, checked)
            if ref is None:
                ref = (dl, dr, sub)
                continue
            assert np.array_equal(dl, ref[0]) and np.array_equal(dr, ref[1]), (cdt, checked)
            assert np.array_equal(np.isnan(sub), np.isnan(ref[2])), (cdt, checked)
            ok = ~np.isnan(ref[2])
            assert np.array_equal(sub[ok].view(np.uint32), ref[2][ok].view(np.uint32)), (cdt, checked)
