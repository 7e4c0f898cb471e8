"""GPU parity of the soft-argmin variant (forward, hand-written backward, L1
loss) against the FP64 oracle, whose own gradient is pinned by central
finite differences (tests/test_oracle_soft.py).

Bar: d_soft within 1e-4 px, log-sum-exp within 1e-4; image gradients with
||g_gpu - g_oracle||_2 / ||g_oracle||_2 <= 1e-3 (maximum element error
reported).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402

GRAD_RTOL = 1e-3


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    st.lib()
    return torch.device("cuda:0")


def _crop_pair(seed, y0, x0, H, W, shift=3):
    Lrgb, Rrgb, gt = synth.tissue_pair(seed, 320, 180, 2.0, 14.0)
    L = oracle.gray(Lrgb)[y0:y0 + H, x0:x0 + W].astype(np.float64)
    R = oracle.gray(Rrgb)[y0:y0 + H, x0:x0 + W].astype(np.float64)
    return L, R, gt[y0:y0 + H, x0:x0 + W]


def _handle(H, W, D, B=1):
    p = st.stereo_default_params(max_width=W, max_height=H, num_disp=D, soft_argmin=1)
    return st.stereo_create(p)


def _T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)


@pytest.mark.parametrize("r,D,tau", [(5, 16, 0.1), (2, 9, 0.05), (7, 24, 0.3)])
def test_forward_matches_oracle(dev, r, D, tau):
    L, R, gt = _crop_pair(synth.seed_for(4), 40, 60, 64, 80)
    ds_ref, lse_ref, hv = oracle.softargmin_fwd(L, R, 0, D, r, tau)
    h = _handle(64, 80, D)
    ds = torch.empty((64, 80), dtype=torch.float32, device=dev)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, _T(L, dev), _T(R, dev), 0, D, r, tau, ds, lse)
    torch.cuda.synchronize()
    ds, lse = ds.cpu().numpy(), lse.cpu().numpy()
    assert np.array_equal(np.isnan(ds), ~hv)
    assert np.max(np.abs(ds[hv] - ds_ref[hv])) <= 1e-4
    assert np.max(np.abs(lse[hv] - lse_ref[hv]) / np.maximum(1.0, np.abs(lse_ref[hv]))) <= 1e-5
    h.close()


@pytest.mark.parametrize("D,H,W", [(16, 64, 80), (100, 40, 200), (150, 40, 232)])
@pytest.mark.parametrize("tau", [0.02, 0.005, 0.001])
def test_forward_small_temperature(dev, D, H, W, tau):
    """Temperatures below 0.025 (weights relative to each pixel's best
    candidate, in the cost kernel's forward form for D <= 128 and in the
    volume kernel above): d_soft and the log-sum-exp against the oracle.
    FP32 ZNCC values carry up to ~1e-6 of error, which moves a weight by
    ~1e-6 / tau relative, so the d_soft bar is 1e-4 + 4e-6 / tau * D px and
    the log-sum-exp's 1e-5 relative + 2e-7 / tau; as
    tau -> 0 d_soft tends to the winner-take-all disparity where the best
    candidate leads the second by more than 20 tau (Sec. II-A winners)."""
    L, R, gt = _crop_pair(synth.seed_for(4), 30, 40, H, W)
    ds_ref, lse_ref, hv = oracle.softargmin_fwd(L, R, 0, D, 5, tau)
    h = _handle(H, W, D)
    ds = torch.empty((H, W), dtype=torch.float32, device=dev)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, _T(L, dev), _T(R, dev), 0, D, 5, tau, ds, lse)
    torch.cuda.synchronize()
    ds, lse = ds.cpu().numpy(), lse.cpu().numpy()
    h.close()
    assert np.array_equal(np.isnan(ds), ~hv)
    err = np.abs(ds[hv] - ds_ref[hv])
    print(f"tau {tau}: max |d_soft - oracle| {err.max():.2e} px")
    assert err.max() <= 1e-4 + 4e-6 / tau * D
    # the log-sum-exp is about max(rho) / tau: an FP32 rho error of ~1e-7
    # moves it by ~1e-7 / tau
    lerr = np.abs(lse[hv] - lse_ref[hv]) - 1e-5 * np.maximum(1.0, np.abs(lse_ref[hv]))
    assert np.max(lerr) <= 2e-7 / tau
    if tau <= 0.001:
        m = oracle.match(np.clip(np.rint(L), 0, 255).astype(np.uint8), np.clip(np.rint(R), 0, 255).astype(np.uint8),
                         0, D, 5)
        clear = hv & (m["gapL"] > 20 * tau) & (m["dL"] != oracle.INVALID)
        assert clear.sum() > 100
        assert np.max(np.abs(ds[clear] - m["dL"][clear])) <= 0.01


def test_backward_small_temperature(dev):
    """tau = 0.01: the backward pass uses the log-sum-exp of the shifted
    forward; image gradients against the oracle's."""
    H, W, D, r, tau = 48, 200, 100, 5, 0.01
    L, R, gt = _crop_pair(synth.seed_for(4, 1), 30, 100, H, W)
    rng = np.random.default_rng(12)
    ds_ref, lse_ref, hv = oracle.softargmin_fwd(L, R, 0, D, r, tau)
    g = np.where(hv, rng.normal(0, 1, (H, W)), 0.0)
    gL_ref, gR_ref = oracle.softargmin_bwd(L, R, 0, D, r, tau, g)
    h = _handle(H, W, D)
    tL, tR = _T(L, dev), _T(R, dev)
    ds = torch.empty((H, W), dtype=torch.float32, device=dev)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, tL, tR, 0, D, r, tau, ds, lse)
    gL, gR = torch.empty_like(ds), torch.empty_like(ds)
    st.stereo_softargmin_bwd(h, tL, tR, 0, D, r, tau, ds, lse, _T(g, dev), gL, gR)
    torch.cuda.synchronize()
    h.close()
    for got, ref in ((gL.cpu().numpy(), gL_ref), (gR.cpu().numpy(), gR_ref)):
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"tau {tau}: grad rel L2 {rel:.2e}")
        assert rel <= GRAD_RTOL


def test_forward_two_chunks_matches_oracle(dev):
    """num_disp > 128: the forward reads the FP32 volume (two disparity
    chunks) instead of summing inside the cost kernel."""
    H, W, D, r, tau = 40, 232, 150, 3, 0.1
    L, R, gt = _crop_pair(synth.seed_for(4), 30, 40, H, W)
    ds_ref, lse_ref, hv = oracle.softargmin_fwd(L, R, 0, D, r, tau)
    assert hv.sum() > 1000
    h = _handle(H, W, D)
    ds = torch.empty((H, W), dtype=torch.float32, device=dev)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, _T(L, dev), _T(R, dev), 0, D, r, tau, ds, lse)
    torch.cuda.synchronize()
    ds, lse = ds.cpu().numpy(), lse.cpu().numpy()
    assert np.array_equal(np.isnan(ds), ~hv)
    assert np.max(np.abs(ds[hv] - ds_ref[hv])) <= 1e-4
    assert np.max(np.abs(lse[hv] - lse_ref[hv]) / np.maximum(1.0, np.abs(lse_ref[hv]))) <= 1e-5
    h.close()


@pytest.mark.parametrize("r,D,H,W,d_min", [
    (5, 16, 64, 64, 0), (3, 12, 64, 64, 0),
    (7, 40, 50, 70, 0),      # K = 2: two disparity chunks, ragged last run
    (1, 33, 48, 45, 0),
    (5, 100, 48, 200, 0),    # K = 4, one chunk of 128 with 28 lanes' candidates beyond D
    (7, 128, 40, 220, 0),    # K = 4, all 128 candidates of the batch form's range (r = 7)
    (5, 128, 24, 200, 0),    # the differentiation workload's D = 128, r = 5
    (5, 128, 30, 210, -6),   # K = 4 with a negative first disparity
    (3, 150, 32, 212, 0)])   # D > 128: through the FP32 volume
def test_backward_matches_oracle_gradient(dev, r, D, H, W, d_min):
    """Crop of a tissue pair, candidates d_min..d_min+D-1, tau = 0.1, random
    upstream gradient.  The crops are wide enough that pixels near the right
    edge have every candidate valid.  Forward compared element by element on
    the same crop."""
    tau = 0.1
    L, R, gt = _crop_pair(synth.seed_for(4, 1), 30, 100, H, W)
    rng = np.random.default_rng(11)
    ds_ref, lse_ref, hv = oracle.softargmin_fwd(L, R, d_min, D, r, tau)
    assert hv.sum() > 200
    g = np.where(hv, rng.normal(0, 1, (H, W)), 0.0)
    gL_ref, gR_ref = oracle.softargmin_bwd(L, R, d_min, D, r, tau, g)
    h = _handle(H, W, D)
    tL, tR = _T(L, dev), _T(R, dev)
    ds = torch.empty((H, W), dtype=torch.float32, device=dev)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, tL, tR, d_min, D, r, tau, ds, lse)
    gL = torch.empty_like(ds)
    gR = torch.empty_like(ds)
    st.stereo_softargmin_bwd(h, tL, tR, d_min, D, r, tau, ds, lse, _T(g, dev), gL, gR)
    torch.cuda.synchronize()
    dsn, lsen = ds.cpu().numpy(), lse.cpu().numpy()
    assert np.array_equal(np.isnan(dsn), ~hv)
    assert np.max(np.abs(dsn[hv] - ds_ref[hv])) <= 1e-4
    assert np.max(np.abs(lsen[hv] - lse_ref[hv]) / np.maximum(1.0, np.abs(lse_ref[hv]))) <= 1e-5
    for got, ref in ((gL.cpu().numpy(), gL_ref), (gR.cpu().numpy(), gR_ref)):
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"grad rel L2 {rel:.2e}, max abs err {np.max(np.abs(got - ref)):.2e} (max |g| {np.max(np.abs(ref)):.2e})")
        assert rel <= GRAD_RTOL
    h.close()


@pytest.mark.parametrize("r,tau", [(1, 0.1), (1, 0.01), (5, 0.1), (5, 0.01), (1, 0.001), (7, 0.001)])
def test_flat_patches_of_float_images(dev, r, tau):
    """Float images with non-integer values (the gray crop / 255) and
    constant patches in the left one.  A patch's windows have zero variance:
    the oracle's sums are exact and give 0; the FP32 sums leave a rounding
    residue (once a denormal, whose reciprocal square root made the forward
    infinite and the gradients NaN), which the preparation kernel now reads
    as zero variance.  Forward and gradients finite everywhere, and at the
    pixels whose left window lies inside a patch (rho = 0 for every
    candidate) d_soft equal to the oracle's.  Elsewhere such low-texture
    non-integer windows carry the FP32 limit of B = N SS - S^2 (relative
    error about N 2^-24 SS / var), so the element-wise bars of the
    integer-valued crops above do not apply."""
    H, W, D = 48, 96, 16
    L, R, gt = _crop_pair(synth.seed_for(4, 2), 20, 80, H, W)
    L = (L / 255.0).astype(np.float32).astype(np.float64)
    R = (R / 255.0).astype(np.float32).astype(np.float64)
    L[12:30, 30:60] = L[12, 30]                       # a flat patch
    L[36:44, 70:90] = np.float32(1.0 / 3.0)          # and one at a non-representable third
    ds_ref, lse_ref, hv = oracle.softargmin_fwd(L, R, 0, D, r, tau)
    inside = np.zeros((H, W), bool)
    inside[12 + r:30 - r, 30 + r:60 - r] = True
    inside[36 + r:44 - r, 70 + r:90 - r] = True
    g = np.where(hv, np.random.default_rng(3).normal(0, 1, (H, W)), 0.0)
    h = _handle(H, W, D)
    tL, tR = _T(L, dev), _T(R, dev)
    ds = torch.empty((H, W), dtype=torch.float32, device=dev)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, tL, tR, 0, D, r, tau, ds, lse)
    gL, gR = torch.empty_like(ds), torch.empty_like(ds)
    st.stereo_softargmin_bwd(h, tL, tR, 0, D, r, tau, ds, lse, _T(g, dev), gL, gR)
    torch.cuda.synchronize()
    dsn, lsen = ds.cpu().numpy(), lse.cpu().numpy()
    assert np.array_equal(np.isnan(dsn), ~hv)
    assert np.all(np.isfinite(lsen[hv]))
    flat = inside & hv
    if flat.any():
        assert np.max(np.abs(dsn[flat] - ds_ref[flat])) <= 1e-4
    assert np.all(np.isfinite(gL.cpu().numpy())) and np.all(np.isfinite(gR.cpu().numpy()))
    h.close()


@pytest.mark.parametrize("r,tau", [(1, 0.1), (5, 0.1), (5, 0.01), (7, 0.1)])
def test_nearly_flat_windows_of_integer_images(dev, r, tau):
    """Integer-valued images (the 8-bit gray crop) with constant patches in
    which single pixels sit one or two levels off: those windows have a small
    but exact nonzero variance (B = N SS - S^2 >= N - 1 in integers) and a
    well-defined ZNCC, which the FP32 sums of integer pixels compute exactly.
    Their d_soft, log-sum-exp and gradients must match the oracle everywhere
    (a variance floor meant for the rounding residue of non-integer sums once
    zeroed them: rho = 0 for every candidate and d_soft off by tens of
    pixels)."""
    H, W, D = 48, 112, 24
    L, R, gt = _crop_pair(synth.seed_for(4, 3), 20, 80, H, W)
    L[10:34, 20:70] = L[10, 20]
    L[10:34:7, 25:70:9] += 1.0                      # sparse one-level bumps
    L[22, 40] += 2.0
    R[10:34, 10:60] = R[10, 10]
    R[14:34:6, 15:60:11] -= 1.0
    L, R = np.clip(L, 0, 255), np.clip(R, 0, 255)
    ds_ref, lse_ref, hv = oracle.softargmin_fwd(L, R, 0, D, r, tau)
    g = np.where(hv, np.random.default_rng(4).normal(0, 1, (H, W)), 0.0)
    gL_ref, gR_ref = oracle.softargmin_bwd(L, R, 0, D, r, tau, g)
    h = _handle(H, W, D)
    tL, tR = _T(L, dev), _T(R, dev)
    ds = torch.empty((H, W), dtype=torch.float32, device=dev)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, tL, tR, 0, D, r, tau, ds, lse)
    gL, gR = torch.empty_like(ds), torch.empty_like(ds)
    st.stereo_softargmin_bwd(h, tL, tR, 0, D, r, tau, ds, lse, _T(g, dev), gL, gR)
    torch.cuda.synchronize()
    dsn, lsen = ds.cpu().numpy(), lse.cpu().numpy()
    assert np.array_equal(np.isnan(dsn), ~hv)
    assert np.max(np.abs(dsn[hv] - ds_ref[hv])) <= 1e-4
    assert np.max(np.abs(lsen[hv] - lse_ref[hv]) / np.maximum(1.0, np.abs(lse_ref[hv]))) <= 1e-5
    for got, ref in ((gL.cpu().numpy(), gL_ref), (gR.cpu().numpy(), gR_ref)):
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= GRAD_RTOL
    h.close()


def test_l1_loss_many_partial_sums(dev):
    """Three 960x540 maps (1.55 M values, the largest number of partial sums)
    with a tenth of the pixels without a valid candidate: loss and gradient
    against the oracle."""
    rng = np.random.default_rng(3)
    shape = (3, 540, 960)
    ds = rng.uniform(0, 128, shape).astype(np.float32)
    ds[rng.random(shape) < 0.1] = np.nan
    gt = rng.uniform(0, 128, shape).astype(np.float32)
    hv = ~np.isnan(ds)
    h = _handle(32, 32, 16)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    g = torch.empty(shape, dtype=torch.float32, device=dev)
    st.stereo_l1_loss(h, _T(ds, dev), _T(gt, dev), loss, g)
    torch.cuda.synchronize()
    loss_ref, g_ref = oracle.l1_loss(np.where(hv, ds, 0).astype(np.float64), hv, gt)
    assert abs(loss.item() - loss_ref) <= 1e-5 * max(1.0, loss_ref)
    kinks = np.abs(ds.astype(np.float64) - gt) == 0
    assert np.all((g.cpu().numpy() == g_ref.astype(np.float32)) | kinks)
    h.close()


def test_autograd_l1_loss(dev):
    """torch.autograd through SoftArgminZNCC with the library's L1 loss
    reproduces the oracle's loss and gradients (batch of two crops)."""
    H, W, D, r, tau = 48, 64, 16, 5, 0.1
    crops = [_crop_pair(synth.seed_for(4, b), 50, 120, H, W) for b in range(2)]
    L = np.stack([c[0] for c in crops])
    R = np.stack([c[1] for c in crops])
    gt = np.stack([c[2] for c in crops])
    h = _handle(H, W, D)
    tL = _T(L, dev).requires_grad_(True)
    tR = _T(R, dev).requires_grad_(True)
    ds = st.soft_argmin(tL, tR, h, 0, D, r, tau)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    g = torch.empty_like(ds)
    st.stereo_l1_loss(h, ds.detach(), _T(gt, dev), loss, g)
    ds.backward(g)
    torch.cuda.synchronize()
    # oracle: both crops, one mean over all valid pixels
    refs = [oracle.softargmin_fwd(L[b], R[b], 0, D, r, tau) for b in range(2)]
    ds_ref = np.stack([x[0] for x in refs])
    hv = np.stack([x[2] for x in refs])
    loss_ref, g_ref = oracle.l1_loss(ds_ref, hv, gt)
    assert abs(loss.item() - loss_ref) <= 1e-4 * max(1.0, loss_ref)
    kinks = np.abs(ds_ref - gt) < 1e-3            # sign may differ at |e| ~ 0
    g_gpu = g.cpu().numpy()
    assert np.all((g_gpu == g_ref.astype(np.float32)) | kinks | ~hv)
    for b in range(2):
        gl_ref, gr_ref = oracle.softargmin_bwd(L[b], R[b], 0, D, r, tau, g_gpu[b].astype(np.float64))
        for got, ref in ((tL.grad[b].cpu().numpy(), gl_ref), (tR.grad[b].cpu().numpy(), gr_ref)):
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= GRAD_RTOL
    h.close()


def test_full_size_batch_sampled(dev):
    """Two 960x540 pairs (the batch form uses 8), D = 128, tau = 0.1: forward
    sampled against the oracle pixel by pixel; gradients finite."""
    B, H, W, D, r, tau = 2, 540, 960, 128, 5, 0.1
    pairs = [synth.tissue_pair(synth.seed_for(4, b)) for b in range(B)]
    L = np.stack([oracle.gray(p[0]) for p in pairs]).astype(np.float32)
    R = np.stack([oracle.gray(p[1]) for p in pairs]).astype(np.float32)
    h = _handle(H, W, D)
    tL, tR = _T(L, dev), _T(R, dev)
    ds = torch.empty((B, H, W), dtype=torch.float32, device=dev)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, tL, tR, 0, D, r, tau, ds, lse)
    g = torch.randn_like(ds).nan_to_num(0) * (~torch.isnan(ds))
    gL, gR = torch.empty_like(ds), torch.empty_like(ds)
    st.stereo_softargmin_bwd(h, tL, tR, 0, D, r, tau, ds, lse, g, gL, gR)
    torch.cuda.synchronize()
    assert torch.isfinite(gL).all() and torch.isfinite(gR).all()
    ds_np = ds.cpu().numpy()
    rng = np.random.default_rng(3)
    for _ in range(12):
        b, y, x = int(rng.integers(0, B)), int(rng.integers(5, H - 5)), int(rng.integers(140, W - 6))
        # the crop holds every window of pixel (x, y) and of all its candidates
        win = (slice(y - 5, y + 6), slice(x - 132, x + 6))
        ref, _, hv = oracle.softargmin_fwd(L[b][win].astype(np.float64), R[b][win].astype(np.float64),
                                           0, D, r, tau)
        assert hv[5, 132] and abs(ds_np[b, y, x] - ref[5, 132]) <= 1e-4
    h.close()
