"""GPU parity of the ZNCC / winner-take-all / sub-pixel / left-right stage
(Sec. II-A) against the FP64 oracle, on the same seeded inputs.

Bar: integer disparities bit-exact except where the oracle's two best ZNCC
values differ by less than 1e-5; cost volume (FP32) within 1e-6 of the FP64
ZNCC; sub-pixel within 0.01 px.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import NEAR_TIE, SUB_TOL, to_np, int_map_mismatch, describe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    st.lib()
    return torch.device("cuda:0")


def run_stage_match(dev, L, R, d_min, D, r, cdt=st.COST_F32, sampling=st.SAMPLE_FULL):
    H, W = L.shape
    p = st.stereo_default_params(max_width=W, max_height=H, num_disp=D, d_min=d_min, win_radius=r,
                                 cost_dtype=cdt, sampling=sampling)
    h = st.stereo_create(p)
    tL = torch.from_numpy(np.ascontiguousarray(L)).to(dev)
    tR = torch.from_numpy(np.ascontiguousarray(R)).to(dev)
    dl = torch.empty((H, W), dtype=torch.int16, device=dev)
    dr = torch.empty_like(dl)
    sub = torch.empty((H, W), dtype=torch.float32, device=dev)
    cost = None
    if cdt != st.COST_NONE:
        tdt = {st.COST_F32: torch.float32, st.COST_F16: torch.float16, st.COST_BF16: torch.bfloat16}[cdt]
        # zero-filled: the library itself must write NaN for invalid candidates
        cost = torch.zeros((H, W, st.cost_stride(D)), dtype=tdt, device=dev)
    st.stereo_stage_match(h, tL, tR, d_min, D, r, sampling, cdt, dl, dr, sub, cost)
    torch.cuda.synchronize()
    assert st.stereo_get_device_error(h) == 0
    h.close()
    out = dict(dL=to_np(dl), dR=to_np(dr), sub=to_np(sub))
    if cost is not None:
        out["cost"] = to_np(cost.float())[:, :, :D]
    return out


def check_against_oracle(g, m, D, sub_check=True):
    exemptL = m["gapL"] < NEAR_TIE
    bad = int_map_mismatch(g["dL"], m["dL"], exemptL)
    assert len(bad) == 0, "left WTA mismatch " + describe(bad, g["dL"], m["dL"], m["gapL"])
    exemptR = m["gapR"] < NEAR_TIE
    bad = int_map_mismatch(g["dR"], m["dR"], exemptR)
    assert len(bad) == 0, "right WTA mismatch " + describe(bad, g["dR"], m["dR"], m["gapR"])
    if sub_check:
        same = (g["dL"] == m["dL"]) & (m["dL"] != oracle.INVALID)
        err = np.abs(g["sub"][same] - m["sub"][same])
        assert np.all(err <= SUB_TOL), f"sub-pixel max err {err.max()}"
        inv = m["dL"] == oracle.INVALID
        assert np.all(np.isnan(g["sub"][inv]))


@pytest.mark.parametrize("shape,d_min,D,r", [
    ((23, 37), 0, 5, 1),
    ((23, 37), -3, 7, 2),
    ((40, 61), 0, 33, 3),       # two disparity chunks of 32
    ((35, 90), 2, 64, 4),       # K = 2
    ((30, 150), 0, 100, 5),     # K = 4, ragged D
    ((26, 230), -20, 150, 5),   # two chunks of 128, negative d_min
    ((33, 80), 0, 16, 7),
    ((30, 260), 0, 192, 6),     # 128 disparities at K = 4, then 64 at K = 2
])
def test_random_pairs_small(dev, shape, d_min, D, r):
    rng = np.random.default_rng(hash((shape, d_min, D, r)) & 0xFFFF)
    H, W = shape
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    g = run_stage_match(dev, L, R, d_min, D, r)
    m = oracle.match(L, R, d_min, D, r)
    check_against_oracle(g, m, D)
    cv = oracle.cost_volume(L, R, d_min, D, r)
    assert np.array_equal(np.isnan(g["cost"]), np.isnan(cv))
    ok = ~np.isnan(cv)
    assert np.max(np.abs(g["cost"][ok] - cv[ok])) <= 1e-6


def test_binary_images_extreme_window_sums(dev):
    """Pixels of 0 and 255 only, 15x15 windows: the window sums of products
    of the integer cost form reach their largest magnitudes (every shifted
    product is +-128*127 or 127^2 or 128^2), where an inexact sum would show."""
    rng = np.random.default_rng(11)
    L = (rng.integers(0, 2, (36, 120)) * 255).astype(np.uint8)
    R = np.roll(L, -9, axis=1)
    R[:, -12:] = (rng.integers(0, 2, (36, 12)) * 255).astype(np.uint8)
    g = run_stage_match(dev, L, R, 0, 40, 7)
    m = oracle.match(L, R, 0, 40, 7)
    check_against_oracle(g, m, 40)
    cv = oracle.cost_volume(L, R, 0, 40, 7)
    ok = ~np.isnan(cv)
    assert np.array_equal(np.isnan(g["cost"]), np.isnan(cv))
    assert np.max(np.abs(g["cost"][ok] - cv[ok])) <= 1e-6
    assert np.mean(g["dL"][7:-7, 30:-7] == 9) > 0.95          # the shift is found


def test_perlin_pair_full(dev):
    """The 320x240 Perlin workload (D = 32, 11x11 window), every pixel."""
    L, R, gt = synth.perlin_pair(synth.seed_for(0))
    g = run_stage_match(dev, L, R, 0, 32, 5)
    m = oracle.match(L, R, 0, 32, 5)
    check_against_oracle(g, m, 32)


def test_images_smaller_than_window(dev):
    rng = np.random.default_rng(5)
    L = rng.integers(0, 256, (9, 9), dtype=np.uint8)
    g = run_stage_match(dev, L, L.copy(), 0, 4, 5)
    assert np.all(g["dL"] == oracle.INVALID) and np.all(g["dR"] == oracle.INVALID)
    assert np.all(np.isnan(g["sub"]))


def test_constant_and_degenerate_windows(dev):
    """Constant windows have ZNCC 0 for every candidate: the smallest valid d
    wins, exactly as in the oracle."""
    H, W = 30, 60
    L = np.full((H, W), 90, np.uint8)
    L[:, 30:] = np.random.default_rng(1).integers(0, 256, (H, 30), dtype=np.uint8)
    R = np.roll(L, -3, axis=1)
    g = run_stage_match(dev, L, R, 0, 12, 3)
    m = oracle.match(L, R, 0, 12, 3)
    check_against_oracle(g, m, 12)


def test_half_precision_cost_storage(dev):
    """FP16 / BF16 cost storage: the winners are unchanged (decided in FP32),
    the sub-pixel disparities too (their three costs are recomputed in FP32);
    the stored costs are within the storage format's rounding."""
    L, R, gt = synth.perlin_pair(synth.seed_for(0))
    L, R = L[:80], R[:80]
    m = oracle.match(L, R, 0, 32, 5)
    cv = oracle.cost_volume(L, R, 0, 32, 5)
    ok = ~np.isnan(cv)
    for cdt, eps in ((st.COST_F16, 2 ** -11), (st.COST_BF16, 2 ** -8)):
        g = run_stage_match(dev, L, R, 0, 32, 5, cdt)
        check_against_oracle(g, m, 32)
        # storage rounding (relative eps) on top of the FP32 computation of
        # c = 1 - rho (absolute ~1e-7)
        err = np.abs(g["cost"][ok] - cv[ok])
        assert np.all(err <= eps * np.abs(cv[ok]) + 3e-7)
        assert np.array_equal(np.isnan(g["cost"]), np.isnan(cv))


@pytest.mark.parametrize("shape,d_min,D,r", [((72, 200), 0, 64, 5), ((90, 240), -8, 128, 7),
                                             ((61, 173), 3, 100, 3), ((40, 300), -20, 128, 1),
                                             # several chunks; winners on both sides of index 128
                                             ((90, 240), -120, 192, 7), ((72, 300), -124, 256, 5),
                                             ((61, 173), -125, 160, 3)])
def test_subpixel_in_cost_kernel_matches_finalize(dev, shape, d_min, D, r):
    """Without an FP32 volume (FP16, BF16 or none) the integer cost kernel
    parks each row's FP32 costs in shared memory: with the whole range in one
    chunk it fits the parabola itself; with several chunks each keeps its own
    winner's three costs (+inf for a neighbour in the other chunk, which the
    finalize kernel then recomputes) and the finalize kernel takes the final
    winner's.  With an FP32 volume the finalize kernel reads the three costs
    back.  All are the same FP32 operations on the same values: winners and
    sub-pixel disparities bit-identical across the four storage types (NaN
    at the same pixels), and within the bar against the oracle."""
    H, W = shape
    L, R, gt = synth.tissue_pair(synth.seed_for(11, D + r), 320, 180, 2.0, 14.0)
    L, R = oracle.gray(L)[:H, :W], oracle.gray(R)[:H, :W]
    ref = run_stage_match(dev, L, R, d_min, D, r, st.COST_F32)
    m = oracle.match(L, R, d_min, D, r)
    check_against_oracle(ref, m, D)
    for cdt in (st.COST_F16, st.COST_BF16, st.COST_NONE):
        g = run_stage_match(dev, L, R, d_min, D, r, cdt)
        assert np.array_equal(g["dL"], ref["dL"]) and np.array_equal(g["dR"], ref["dR"])
        assert np.array_equal(np.isnan(g["sub"]), np.isnan(ref["sub"]))
        ok = ~np.isnan(ref["sub"])
        assert np.array_equal(g["sub"][ok].view(np.uint32), ref["sub"][ok].view(np.uint32))


def test_deterministic(dev):
    L, R, gt = synth.perlin_pair(synth.seed_for(0))
    a = run_stage_match(dev, L, R, 0, 32, 5)
    b = run_stage_match(dev, L, R, 0, 32, 5)
    for k in ("dL", "dR"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["sub"], b["sub"], equal_nan=True)
    assert np.array_equal(a["cost"], b["cost"], equal_nan=True)


@pytest.mark.parametrize("shape,d_min,D,r,cdt", [
    ((23, 37), 0, 5, 1, st.COST_F32),
    ((40, 61), -3, 33, 3, st.COST_F32),
    ((30, 150), 0, 100, 5, st.COST_F16),
    ((26, 230), -20, 100, 5, st.COST_NONE),
    ((33, 80), 0, 16, 7, st.COST_BF16),
])
def test_chessboard_sampling(dev, shape, d_min, D, r, cdt):
    """CHESSBOARD sampling (Sec. II-A: only window offsets with dx + dy even,
    centre included): winners, sub-pixel and the stored volume against the
    oracle's chessboard ZNCC."""
    rng = np.random.default_rng(hash((shape, d_min, D, r, 7)) & 0xFFFF)
    H, W = shape
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    g = run_stage_match(dev, L, R, d_min, D, r, cdt, sampling=st.SAMPLE_CHESSBOARD)
    m = oracle.match(L, R, d_min, D, r, sampling=oracle.SAMPLE_CHESSBOARD)
    check_against_oracle(g, m, D)
    if cdt != st.COST_NONE:
        cv = oracle.cost_volume(L, R, d_min, D, r, sampling=oracle.SAMPLE_CHESSBOARD)
        assert np.array_equal(np.isnan(g["cost"]), np.isnan(cv))
        ok = ~np.isnan(cv)
        eps = {st.COST_F32: 0.0, st.COST_F16: 2 ** -11, st.COST_BF16: 2 ** -8}[cdt]
        assert np.all(np.abs(g["cost"][ok] - cv[ok]) <= eps * np.abs(cv[ok]) + 1e-6)


def test_chessboard_differs_from_full(dev):
    """The two samplings are different windows (guards against the option
    being ignored)."""
    L, R, gt = synth.perlin_pair(synth.seed_for(0))
    L, R = L[:60], R[:60]
    a = run_stage_match(dev, L, R, 0, 32, 5, sampling=st.SAMPLE_CHESSBOARD)
    b = run_stage_match(dev, L, R, 0, 32, 5)
    assert np.nanmax(np.abs(a["cost"] - b["cost"])) > 1e-3
