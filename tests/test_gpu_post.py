"""GPU parity of the left-right check, outlier removal, hole filling
(Sec. II-B) and the improved Laplacian refinement (Sec. II-C), stage by stage:
each GPU stage is fed the oracle's input for that stage.

Bar: integer maps bit-exact; refined disparities within 1e-4 relative, with
the fraction of pixels beyond it reported (the o-update is an argmin whose
near-ties FP32 may break differently from FP64).
"""
import numpy as np
import pytest

import oracle
import synth
from parity import REFINE_RTOL, to_np, int_map_mismatch, describe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402

INV = oracle.INVALID


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    st.lib()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def perlin_stages():
    L, R, gt = synth.perlin_pair(synth.seed_for(0))
    p = oracle.Params(d_min=0, num_disp=32, win_radius=5, smooth_radius=2, smooth_iters=5)
    out = oracle.pipeline(L, R, p)
    return L, R, p, out


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def test_lr_check(dev, perlin_stages):
    L, R, p, o = perlin_stages
    out = torch.empty(L.shape, dtype=torch.int16, device=dev)
    st.stereo_stage_lr(T(o["dL"], dev), T(o["dR"], dev), 1, out)
    assert np.array_equal(to_np(out), o["o_lr"])


def _random_map(rng, H, W, lo, hi, p_inv):
    base = rng.integers(lo, hi, (H, W)).astype(np.int16)
    smooth = np.cumsum(rng.integers(-1, 2, (H, W)), axis=1).astype(np.int16) // 3 + 20
    m = np.where(rng.random((H, W)) < 0.7, smooth, base).astype(np.int16)
    m[rng.random((H, W)) < p_inv] = INV
    return m


def _handle(H, W):
    return st.stereo_create(st.stereo_default_params(max_width=W, max_height=H, num_disp=32))


@pytest.mark.parametrize("radius", [0, 1, 3, 10, 20, 30, 33, 63, 64, 70])
def test_outlier(dev, radius):
    """Radii up to 64 run the line-bitmask test, larger ones the ray walk."""
    rng = np.random.default_rng(radius)
    m = _random_map(rng, 70, 150, 0, 60, 0.15)
    out = torch.empty_like(T(m, dev))
    st.stereo_stage_outlier(_handle(*m.shape), T(m, dev), radius, 2.5, out)
    want = oracle.outlier_removal(m, radius, 2.5)
    bad = int_map_mismatch(to_np(out), want)
    assert len(bad) == 0, describe(bad, to_np(out), want)


@pytest.mark.parametrize("radius,min_dirs", [(50, 4), (5, 2), (50, 8), (63, 3), (70, 4), (1, 1)])
def test_fill_radial(dev, radius, min_dirs):
    """Radii up to 63 run the line-bitmask search, larger ones the ray walk."""
    rng = np.random.default_rng(radius + min_dirs)
    m = _random_map(rng, 64, 130, -10, 60, 0.6)
    out = torch.empty_like(T(m, dev))
    st.stereo_stage_fill_radial(_handle(*m.shape), T(m, dev), radius, min_dirs, out)
    want = oracle.fill_radial(m, radius, min_dirs)
    assert np.array_equal(to_np(out), want)


@pytest.mark.parametrize("radius", [0, 2, 7, 20, 24, 40, 56])
def test_fill_disc(dev, radius):
    rng = np.random.default_rng(100 + radius)
    m = _random_map(rng, 75, 83, -5, 50, 0.55)
    out = torch.empty_like(T(m, dev))
    st.stereo_stage_fill_disc(_handle(*m.shape), T(m, dev), radius, -1, out)
    want = oracle.fill_disc(m, radius)
    assert np.array_equal(to_np(out), want)


def test_fill_disc_sparse_holes(dev):
    """Holes in a few tiles only (a patch, isolated pixels, the image
    corners): tiles without a hole copy their pixels, the others fill from
    windows that reach into hole-free tiles and past the image border."""
    rng = np.random.default_rng(21)
    m = rng.integers(0, 90, (100, 203)).astype(np.int16)
    m[40:52, 70:85] = INV
    m[0, 0] = m[-1, -1] = m[0, -1] = m[-1, 0] = INV
    m[rng.integers(0, 100, 12), rng.integers(0, 203, 12)] = INV
    for radius in (3, 20, 56):
        out = torch.empty_like(T(m, dev))
        st.stereo_stage_fill_disc(_handle(*m.shape), T(m, dev), radius, -1, out)
        want = oracle.fill_disc(m, radius)
        assert np.array_equal(to_np(out), want), radius


def test_fill_disc_wide_rows_large_values(dev):
    """1920-wide rows of disparities near 4300 (the row prefixes wrap around
    32 bits; every disc span stays exact) and negative values."""
    rng = np.random.default_rng(7)
    m = rng.integers(4200, 4352, (12, 1920)).astype(np.int16)
    m[:, :40] = rng.integers(-4096, -4000, (12, 40)).astype(np.int16)
    m[rng.random(m.shape) < 0.3] = INV
    out = torch.empty_like(T(m, dev))
    st.stereo_stage_fill_disc(_handle(*m.shape), T(m, dev), 20, -1, out)
    want = oracle.fill_disc(m, 20)
    assert np.array_equal(to_np(out), want)


def test_postprocess_loop(dev, perlin_stages):
    L, R, p, o = perlin_stages
    H, W = L.shape
    sp = st.stereo_default_params(max_width=W, max_height=H, num_disp=32)
    h = st.stereo_create(sp)
    out = torch.empty((H, W), dtype=torch.int16, device=dev)
    st.stereo_stage_postprocess(h, T(o["o_lr"], dev), out)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(out), o["o_post"])
    h.close()


def _refine_gpu(dev, o_in, cost, L, R, p, cdt=st.COST_F32):
    H, W = o_in.shape
    sp = st.stereo_default_params(max_width=W, max_height=H, num_disp=p.num_disp,
                                  smooth_radius=p.smooth_radius, smooth_iters=p.smooth_iters,
                                  win_radius=p.win_radius)
    h = st.stereo_create(sp)
    d = torch.empty((H, W), dtype=torch.float32, device=dev)
    oo = torch.empty((H, W), dtype=torch.int16, device=dev)
    tc = None
    if cost is not None:
        c = np.full((H, W, st.cost_stride(p.num_disp)), np.nan, np.float32)
        c[:, :, :p.num_disp] = cost
        tc = T(c, dev)
    st.stereo_stage_refine(h, T(o_in, dev), tc, cdt if cost is not None else st.COST_NONE,
                           T(L, dev), T(R, dev), p.d_min, p.num_disp, p.win_radius, d, oo)
    torch.cuda.synchronize()
    h.close()
    return to_np(d), to_np(oo)


def _refine_compare(d_gpu, d_ref, valid):
    assert np.array_equal(np.isnan(d_gpu), ~valid)
    rel = np.abs(d_gpu[valid] - d_ref[valid]) / np.maximum(np.abs(d_ref[valid]), 1.0)
    return rel


def test_refine_stage(dev, perlin_stages):
    L, R, p, o = perlin_stages
    d, oo = _refine_gpu(dev, o["o_post"], o["cost"], L, R, p)
    valid = o["o_post"] != INV
    rel = _refine_compare(d, o["d_final"], valid)
    frac = np.mean(rel > REFINE_RTOL)
    print(f"refine: max rel {rel.max():.3g}, beyond 1e-4: {100 * frac:.3f}% of valid pixels")
    assert frac <= 0.005
    assert np.median(rel) < 1e-6


def test_refine_stage_recomputed_zncc(dev):
    """Without a stored cost volume the o-update recomputes ZNCC directly."""
    L, R, gt = synth.perlin_pair(synth.seed_for(0))
    L, R = L[:60, :120], R[:60, :120]
    p = oracle.Params(d_min=0, num_disp=32, win_radius=5, smooth_radius=2, smooth_iters=3)
    m = oracle.match(L, R, 0, 32, 5)
    o_in = oracle.postprocess(oracle.lr_check(m["dL"], m["dR"]), p)
    d_ref, _ = oracle.refine(o_in, L=L, R=R, p=p)
    d, _ = _refine_gpu(dev, o_in, None, L, R, p)
    rel = _refine_compare(d, d_ref, o_in != INV)
    assert np.mean(rel > REFINE_RTOL) <= 0.005


def test_refine_identities(dev):
    """K = 0 is the identity; a constant map is a fixed point."""
    H, W = 20, 30
    o = np.full((H, W), 12, np.int16)
    o[3:6, 4:9] = INV
    cost = np.full((H, W, 32), 0.5)
    for K in (0, 3):
        p = oracle.Params(num_disp=32, smooth_radius=2, smooth_iters=K)
        d, oo = _refine_gpu(dev, o, cost, o.astype(np.uint8), o.astype(np.uint8), p)
        assert np.all(d[o != INV] == 12.0) and np.all(np.isnan(d[o == INV]))
        assert np.array_equal(oo, o)


@pytest.mark.parametrize("rs", [15, 30])
def test_refine_stage_paper_radius(dev, perlin_stages, rs):
    """Smoothing radius 15 (the paper's) runs the shared-memory tiled path;
    radius 30 exceeds its halo and runs the plain row/column path."""
    L, R, p0, o = perlin_stages
    p = oracle.Params(d_min=0, num_disp=32, win_radius=5, smooth_radius=rs, smooth_iters=5)
    d_ref, _ = oracle.refine(o["o_post"], cost=o["cost"], p=p)
    d, _ = _refine_gpu(dev, o["o_post"], o["cost"], L, R, p)
    rel = _refine_compare(d, d_ref, o["o_post"] != INV)
    print(f"refine rs={rs}: beyond 1e-4: {100 * np.mean(rel > REFINE_RTOL):.3f}%")
    assert np.mean(rel > REFINE_RTOL) <= 0.005
