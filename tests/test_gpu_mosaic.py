"""Point-based TSDF mosaicking on the GPU (Sec. II) against the oracle: two
key frames built from the whole path's output (stereo_match ->
stereo_depth_points), the second seen from a moved camera, then a model
that overflows its capacity.  Bars: every integer decision identical (point
count, which points merged -- their weights -- and the order of appended
points); positions within 1e-5 relative, colours within 1e-3 (FP32 against
FP64 running means)."""
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


def _frame(dev, seed, W=256, H=160):
    Lrgb, Rrgb, gt = synth.tissue_pair(seed, W, H, 6.0, 30.0)
    sp = st.stereo_default_params(max_width=W, max_height=H, num_disp=48, smooth_radius=8)
    h = st.stereo_create(sp)
    dfin = torch.empty((H, W), dtype=torch.float32, device=dev)
    st.stereo_match(h, torch.from_numpy(Lrgb).to(dev), torch.from_numpy(Rrgb).to(dev), disp_final=dfin)
    cam = st.StereoCamera(300.0, W / 2 - 0.5, H / 2 - 0.5, 4.0, 0.0)
    xyz = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    st.stereo_depth_points(dfin, cam, xyz=xyz)
    torch.cuda.synchronize()
    return h, cam, xyz, torch.from_numpy(np.ascontiguousarray(Lrgb)).to(dev)


def _rot_y(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], np.float32)


def _compare(gm, om):
    n = int(gm.count.item())
    assert n == om.count
    wp = gm.wpos[:n].cpu().numpy()
    assert np.array_equal(wp, om.wpos[:n].astype(np.float32))       # integer-valued weights
    pos = gm.pos[:n].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(pos - om.pos[:n]) / np.maximum(np.abs(om.pos[:n]), 1.0)) <= 1e-5
    rgb = gm.rgb[:n].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(rgb - om.rgb[:n])) <= 1e-3
    assert np.max(np.abs(gm.wrgb[:n].cpu().numpy() - om.wrgb[:n])) <= 1e-5


def test_two_frames_against_oracle(dev):
    h, cam, xyz, rgb = _frame(dev, synth.seed_for(6))
    H, W = xyz.shape[:2]
    gm = st.PointModel(4 * W * H, dev)
    om = oracle.PointModel(4 * W * H)
    poses = [(np.eye(3, dtype=np.float32), np.zeros(3, np.float32)),
             (_rot_y(0.02), np.array([0.6, -0.2, 0.3], np.float32))]
    xyz_np = xyz.cpu().numpy()
    img_np = rgb.cpu().numpy()
    for R, t in poses:
        st.stereo_mosaic_frame(h, gm, xyz, rgb, cam, R, t, tau=0.8)
        torch.cuda.synchronize()
        assert oracle.mosaic_frame(om, xyz_np, img_np, cam.f, cam.cx, cam.cy, R, t, 0.8) == 0
        assert int(gm.dropped.item()) == 0
        _compare(gm, om)
    # the second frame merged some points and appended others
    n = om.count
    assert (om.wpos[:n] == 2.0).sum() > 1000 and n > np.isfinite(xyz_np[..., 2]).sum()
    h.close()


def test_capacity_overflow(dev):
    h, cam, xyz, rgb = _frame(dev, synth.seed_for(6, 1), 96, 64)
    cap = 1500
    gm = st.PointModel(cap, dev)
    om = oracle.PointModel(cap)
    I3, Z3 = np.eye(3, dtype=np.float32), np.zeros(3, np.float32)
    st.stereo_mosaic_frame(h, gm, xyz, rgb, cam, I3, Z3, tau=0.5)
    torch.cuda.synchronize()
    dropped = oracle.mosaic_frame(om, xyz.cpu().numpy(), rgb.cpu().numpy(), cam.f, cam.cx, cam.cy, I3, Z3, 0.5)
    assert dropped > 0 and int(gm.dropped.item()) == dropped
    _compare(gm, om)
    h.close()
