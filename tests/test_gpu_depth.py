"""Disparity -> points and normals on the GPU (Sec. II depth from disparity)
against the oracle, on an exact plane and on the refined map of the whole
path.  Bars: the NaN pattern identical; points within 2e-6 relative (FP32
division and products); normals within 1e-3 per component (FP32 central
differences of nearby points)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    st.lib()
    return torch.device("cuda:0")


def _gpu(dev, d32, cam):
    H, W = d32.shape
    xyz = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    nrm = torch.empty_like(xyz)
    st.stereo_depth_points(torch.from_numpy(d32).to(dev), cam, xyz, nrm)
    torch.cuda.synchronize()
    return xyz.cpu().numpy().astype(np.float64), nrm.cpu().numpy().astype(np.float64)


def _compare(g_xyz, g_nrm, r_xyz, r_nrm, nrm_tol=1e-3):
    assert np.array_equal(np.isnan(g_xyz), np.isnan(r_xyz))
    assert np.array_equal(np.isnan(g_nrm), np.isnan(r_nrm))
    ok = ~np.isnan(r_xyz)
    rel = np.abs(g_xyz[ok] - r_xyz[ok]) / np.maximum(np.abs(r_xyz[ok]), 1.0)
    assert rel.max(initial=0) <= 2e-6
    okn = ~np.isnan(r_nrm)
    err = np.abs(g_nrm[okn] - r_nrm[okn]).max(initial=0)
    print(f"points max rel {rel.max(initial=0):.2e}, normals max abs {err:.2e}")
    assert err <= nrm_tol


def test_plane(dev):
    W, H, f, cx, cy, B, doffs = 97, 61, 300.0, 48.0, 30.0, 4.0, 2.5
    n = np.array([0.2, -0.3, -1.0])
    n /= np.linalg.norm(n)
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    ray = np.stack([(u - cx) / f, (v - cy) / f, np.ones_like(u)], -1)
    Z = (n @ np.array([0.0, 0.0, 80.0])) / (ray @ n)
    d32 = (f * B / Z - doffs).astype(np.float32)
    d32[10, 20] = np.nan                            # a hole: its point and 4 normals go NaN
    cam = st.StereoCamera(f, cx, cy, B, doffs)
    g = _gpu(dev, d32, cam)
    r = oracle.depth_points(d32.astype(np.float64), f, cx, cy, B, doffs)
    _compare(*g, *r)
    inner = g[1][1:-1, 1:-1].reshape(-1, 3)
    inner = inner[~np.isnan(inner[:, 0])]
    assert np.max(np.abs(inner - n)) < 1e-3


def test_refined_map_of_the_whole_path(dev):
    """The tissue pair through stereo_match, then its refined map to points."""
    Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(1), 320, 200, 8.0, 40.0)
    H, W = Lrgb.shape[:2]
    sp = st.stereo_default_params(max_width=W, max_height=H, num_disp=64, smooth_radius=15)
    h = st.stereo_create(sp)
    dfin = torch.empty((H, W), dtype=torch.float32, device=dev)
    st.stereo_match(h, torch.from_numpy(Lrgb).to(dev), torch.from_numpy(Rrgb).to(dev), disp_final=dfin)
    torch.cuda.synchronize()
    h.close()
    d32 = dfin.cpu().numpy()
    assert np.isfinite(d32).mean() > 0.5
    f, cx, cy, B = 420.0, W / 2 - 0.5, H / 2 - 0.5, 5.5
    cam = st.StereoCamera(f, cx, cy, B, 0.0)
    g = _gpu(dev, d32, cam)
    r = oracle.depth_points(d32.astype(np.float64), f, cx, cy, B, 0.0)
    _compare(*g, *r)


def test_points_only_and_normals_only(dev):
    d32 = np.full((8, 9), 12.0, np.float32)
    cam = st.StereoCamera(100.0, 4.0, 3.5, 2.0, 0.0)
    t = torch.from_numpy(d32).to(dev)
    xyz = torch.full((8, 9, 3), 7.0, device=dev)
    st.stereo_depth_points(t, cam, xyz=xyz)
    nrm = torch.full((8, 9, 3), 7.0, device=dev)
    st.stereo_depth_points(t, cam, normals=nrm)
    torch.cuda.synchronize()
    r_xyz, r_nrm = oracle.depth_points(d32.astype(np.float64), 100.0, 4.0, 3.5, 2.0)
    assert np.allclose(xyz.cpu().numpy(), r_xyz, rtol=2e-6)
    a = nrm.cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(r_nrm))
    assert np.allclose(a[~np.isnan(a)], r_nrm[~np.isnan(r_nrm)], atol=1e-5)
