"""End-to-end GPU path (stereo_match: gray -> match -> LR -> post -> refine)
against the oracle's whole pipeline on the seeded workloads, and sampled
full-size parity on the 960x540 tissue workload."""
import numpy as np
import pytest

import oracle
import synth
from parity import NEAR_TIE, SUB_TOL, REFINE_RTOL, to_np, int_map_mismatch, describe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402

INV = oracle.INVALID


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    st.lib()
    return torch.device("cuda:0")


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def run_match(dev, Limg, Rimg, p: oracle.Params, cdt=st.COST_F32):
    H, W = Limg.shape[:2]
    sp = st.stereo_default_params(max_width=W, max_height=H, d_min=p.d_min, num_disp=p.num_disp,
                                  win_radius=p.win_radius, cost_dtype=cdt, sampling=p.sampling,
                                  smooth_radius=p.smooth_radius, smooth_iters=p.smooth_iters)
    h = st.stereo_create(sp)
    out = dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
               disp_sub=torch.empty((H, W), dtype=torch.float32, device=dev),
               disp_lr=torch.empty((H, W), dtype=torch.int16, device=dev),
               disp_post=torch.empty((H, W), dtype=torch.int16, device=dev),
               valid=torch.empty((H, W), dtype=torch.uint8, device=dev),
               disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))
    st.stereo_match(h, T(Limg, dev), T(Rimg, dev), **out)
    torch.cuda.synchronize()
    h.close()
    return {k: to_np(v) for k, v in out.items()}


def right_winners(dev, L, R, p: oracle.Params):
    """Right-view winner map from the stage entry point (the cost kernel the
    whole path runs)."""
    H, W = L.shape
    h = st.stereo_create(st.stereo_default_params(max_width=W, max_height=H, d_min=p.d_min,
                                                  num_disp=p.num_disp, win_radius=p.win_radius,
                                                  cost_dtype=st.COST_NONE))
    dl = torch.empty((H, W), dtype=torch.int16, device=dev)
    dr = torch.empty_like(dl)
    sub = torch.empty((H, W), dtype=torch.float32, device=dev)
    st.stereo_stage_match(h, T(L, dev), T(R, dev), p.d_min, p.num_disp, p.win_radius, p.sampling,
                          st.COST_NONE, dl, dr, sub, None)
    torch.cuda.synchronize()
    h.close()
    return to_np(dr)


def test_perlin_end_to_end(dev):
    """320x240, D = 32, 11x11 window, LR check 1 px, hole filling, 5x5
    smoothing (radius 2)."""
    L, R, gt = synth.perlin_pair(synth.seed_for(0))
    p = oracle.Params(d_min=0, num_disp=32, win_radius=5, smooth_radius=2, smooth_iters=5)
    ref = oracle.pipeline(L, R, p)
    m = oracle.match(L, R, 0, 32, 5)
    g = run_match(dev, L, R, p)
    near = m["gapL"] < NEAR_TIE
    bad = int_map_mismatch(g["disp_wta"], ref["dL"], near)
    assert len(bad) == 0, describe(bad, g["disp_wta"], ref["dL"])
    same = (g["disp_wta"] == ref["dL"]) & (ref["dL"] != INV)
    assert np.all(np.abs(g["disp_sub"][same] - ref["sub"][same]) <= SUB_TOL)
    # LR check and post-processing: the oracle's stages on the GPU's own
    # winner maps give the GPU's maps bit for bit (no pixel skipped)
    dR = right_winners(dev, L, R, p)
    bad = int_map_mismatch(dR, m["dR"], m["gapR"] < NEAR_TIE)
    assert len(bad) == 0, describe(bad, dR, m["dR"])
    o_lr = oracle.lr_check(g["disp_wta"], dR, p.lr_thresh)
    assert np.array_equal(g["disp_lr"], o_lr)
    o_post = oracle.postprocess(o_lr, p)
    assert np.array_equal(g["disp_post"], o_post)
    assert np.array_equal(g["valid"].astype(bool), o_post != INV)
    v = ref["o_post"] != INV
    rel = np.abs(g["disp_final"][v] - ref["d_final"][v]) / np.maximum(np.abs(ref["d_final"][v]), 1)
    print(f"end-to-end refine: {100 * np.mean(rel > REFINE_RTOL):.3f}% beyond 1e-4")
    assert np.mean(rel > REFINE_RTOL) <= 0.005
    # accuracy against the generator's field (context): median error < 0.5 px
    gv = g["valid"].astype(bool)
    assert np.median(np.abs(g["disp_final"][gv] - gt[gv])) < 0.5


def test_paper_configuration_chessboard(dev):
    """The paper's own setting (Sec. II-A, Sec. III): chessboard-sampled
    11x11 window, candidates d in [-20, 80), smoothing radius 15, on a
    320x160 tissue crop shifted so that some disparities are negative."""
    Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(1, 5), 320, 160, 4.0, 60.0)
    Lg, Rg = oracle.gray(Lrgb), oracle.gray(Rrgb)
    Lg = np.ascontiguousarray(Lg[:, 10:])          # shift: disparities move by -10
    Rg = np.ascontiguousarray(Rg[:, :-10])
    p = oracle.Params(d_min=-20, num_disp=100, win_radius=5, sampling=oracle.SAMPLE_CHESSBOARD,
                      smooth_radius=15)
    ref = oracle.pipeline(Lg, Rg, p)
    m = oracle.match(Lg, Rg, -20, 100, 5, sampling=oracle.SAMPLE_CHESSBOARD)
    g = run_match(dev, Lg, Rg, p)
    near = m["gapL"] < NEAR_TIE
    bad = int_map_mismatch(g["disp_wta"], ref["dL"], near)
    assert len(bad) == 0, describe(bad, g["disp_wta"], ref["dL"])
    same = (g["disp_wta"] == ref["dL"]) & (ref["dL"] != INV)
    assert np.all(np.abs(g["disp_sub"][same] - ref["sub"][same]) <= SUB_TOL)
    assert (ref["dL"][ref["dL"] != INV] < 0).any()
    v = (ref["o_post"] != INV) & (g["valid"] != 0)
    rel = np.abs(g["disp_final"][v] - ref["d_final"][v]) / np.maximum(np.abs(ref["d_final"][v]), 1)
    print(f"paper configuration: {100 * np.mean(rel > REFINE_RTOL):.3f}% beyond 1e-4")
    assert np.mean(rel > REFINE_RTOL) <= 0.005


def test_tissue_full_size_sampled(dev):
    """960x540 RGB tissue pair, D = 128, full post-processing: every GPU
    winner-take-all pixel of a sample of rows is checked against the oracle
    computed pixel by pixel."""
    Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(1))
    p = oracle.Params(d_min=0, num_disp=128, win_radius=5)
    g = run_match(dev, Lrgb, Rrgb, p)
    Lg, Rg = oracle.gray(Lrgb), oracle.gray(Rrgb)
    rng = np.random.default_rng(7)
    checked = 0
    for _ in range(300):
        y = int(rng.integers(0, 540))
        x = int(rng.integers(0, 960))
        d, gap, sub = oracle.wta_left_pixel(Lg, Rg, 0, 128, 5, x, y)
        if gap < NEAR_TIE:
            continue
        assert g["disp_wta"][y, x] == d, (x, y)
        if d != INV:
            assert abs(g["disp_sub"][y, x] - sub) <= SUB_TOL
        checked += 1
    assert checked > 250
    # properties that hold at any size
    wta = g["disp_wta"]
    assert np.all((wta == INV) | ((wta >= 0) & (wta < 128)))
    fin = g["disp_final"]
    v = g["valid"].astype(bool)
    assert np.all(np.isnan(fin[~v])) and np.all(np.isfinite(fin[v]))
    assert np.all(fin[v] > -6) and np.all(fin[v] < 133)


def test_rgb_and_pitch_inputs(dev):
    """RGB inputs go through the fixed-point gray conversion first."""
    Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(1), 200, 90)
    g_rgb = torch.empty((90, 200), dtype=torch.uint8, device=dev)
    st.stereo_gray(T(Lrgb, dev), g_rgb)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(g_rgb), oracle.gray(Lrgb))


def test_graph_replay_matches_direct_launches(dev):
    """On a non-default stream stereo_match replays a captured CUDA graph;
    its outputs equal those of plain launches, also after the buffers
    change (which captures a new graph)."""
    L, R, gt = synth.perlin_pair(synth.seed_for(0))
    H, W = L.shape
    sp = st.stereo_default_params(max_width=W, max_height=H, num_disp=32, smooth_radius=2)
    h = st.stereo_create(sp)
    tL, tR = T(L, dev), T(R, dev)

    def outs():
        return dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                    disp_post=torch.empty((H, W), dtype=torch.int16, device=dev),
                    disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))

    ref = outs()
    st.stereo_match(h, tL, tR, **ref)           # default stream: plain launches
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    for _ in range(2):
        for trial in range(3):                  # capture, replay, replay
            o = outs() if trial == 0 else o
            with torch.cuda.stream(s):
                st.stereo_match(h, tL, tR, **o, stream=s)
            s.synchronize()
            for k in ref:
                assert torch.equal(o[k].nan_to_num(-1), ref[k].nan_to_num(-1)), k
    h.close()


def test_graph_cache_alternating_buffer_sets(dev):
    """A double-buffered loop alternates two argument sets (two cached
    graphs): every call writes the same maps as plain launches, and the
    launch counter counts each call's kernels once, capturing calls
    included."""
    H, W = 96, 160
    pairs = []
    for i in range(2):
        Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(1, 10 + i), W, H, 2.0, 20.0)
        pairs.append((T(Lrgb, dev), T(Rrgb, dev)))
    sp = st.stereo_default_params(max_width=W, max_height=H, num_disp=32, smooth_radius=4)
    h = st.stereo_create(sp)

    def outs():
        return dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                    disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))

    refs = []
    for tL, tR in pairs:
        o = outs()
        st.stereo_match(h, tL, tR, **o)          # default stream: plain launches
        torch.cuda.synchronize()
        refs.append(o)
    bufs = [outs(), outs()]
    s = torch.cuda.Stream()
    per_call = None
    for it in range(6):
        i = it % 2
        n0 = st.stereo_launch_count()
        with torch.cuda.stream(s):
            st.stereo_match(h, *pairs[i], **bufs[i], stream=s)
        s.synchronize()
        n = st.stereo_launch_count() - n0
        per_call = per_call or n
        assert n == per_call
        for k in refs[i]:
            assert torch.equal(bufs[i][k].nan_to_num(-1), refs[i][k].nan_to_num(-1)), (it, k)
    h.close()
