"""Point-based TSDF mosaicking on the GPU (Sec. II) against the FP64
oracle: key frames built from the whole path's output (stereo_match ->
stereo_depth_points), seen from moved cameras, then a model that overflows
its capacity.

The GPU takes its projection, z-buffer and merge decisions in single
precision, the oracle in double precision.  Before each frame the oracle's
model is set to the GPU's model (so both start from the same points), and
the oracle reports which decisions lie within FP32 reach of an edge
(projection within 2e-3 px of a rounding edge, depth ties within 1e-5
relative, merge tests within 1e-5 relative of the truncation distance).
Outside those, every decision must agree: the weights of the old points,
the set of appended pixels and their row-major order.  Positions within
1e-5 relative, colours within 1e-3 (FP32 against FP64 running means).
"""
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


MARGINS = (2e-3, 1e-5)


def _oracle_from(gm):
    """An oracle model holding the GPU model's current points (float32 values
    widened to float64)."""
    om = oracle.PointModel(gm.capacity)
    n = int(gm.count.item())
    om.pos[:n] = gm.pos[:n].double().cpu().numpy()
    om.rgb[:n] = gm.rgb[:n].double().cpu().numpy()
    om.wpos[:n] = gm.wpos[:n].double().cpu().numpy()
    om.wrgb[:n] = gm.wrgb[:n].double().cpu().numpy()
    om.count = n
    return om


def _pixel_of(P, R, t, cam, W):
    """Pixel index an appended point came from: its camera-frame position is
    the pixel's stereo point, whose projection is the pixel centre."""
    X = P.astype(np.float64) @ R.astype(np.float64).T + t.astype(np.float64)
    u = np.floor(cam.f * X[:, 0] / X[:, 2] + cam.cx + 0.5).astype(np.int64)
    v = np.floor(cam.f * X[:, 1] / X[:, 2] + cam.cy + 0.5).astype(np.int64)
    return v * W + u


def _compare(gm, om, n0, mg, R, t, cam, W):
    fp, fq, src = mg["fragile_pix"].ravel(), mg["fragile_pt"], mg["src_pixel"]
    ng, no = int(gm.count.item()), om.count
    # the points the model held before the frame
    keep = ~fq
    wp = gm.wpos[:n0].cpu().numpy()
    assert np.array_equal(wp[keep], om.wpos[:n0][keep].astype(np.float32))      # integer-valued weights
    pos = gm.pos[:n0].cpu().numpy().astype(np.float64)[keep]
    assert np.max(np.abs(pos - om.pos[:n0][keep]) / np.maximum(np.abs(om.pos[:n0][keep]), 1.0), initial=0) <= 1e-5
    rgb = gm.rgb[:n0].cpu().numpy().astype(np.float64)[keep]
    assert np.max(np.abs(rgb - om.rgb[:n0][keep]), initial=0) <= 1e-3
    assert np.max(np.abs(gm.wrgb[:n0].cpu().numpy()[keep] - om.wrgb[:n0][keep]), initial=0) <= 1e-5
    # appended points: the same pixels outside the marked ones, in row-major order
    gpos = gm.pos[n0:ng].cpu().numpy()
    gpix = _pixel_of(gpos, R, t, cam, W)
    assert np.all(np.diff(gpix) > 0)
    opix = src[n0:no].astype(np.int64)
    only_g = np.setdiff1d(gpix, opix)
    only_o = np.setdiff1d(opix, gpix)
    assert fp[only_g].all() and fp[only_o].all()
    common, ig, io = np.intersect1d(gpix, opix, return_indices=True)
    assert np.max(np.abs(gpos[ig] - om.pos[n0 + io]) / np.maximum(np.abs(om.pos[n0 + io]), 1.0), initial=0) <= 1e-5
    assert np.array_equal(gm.rgb[n0:ng].cpu().numpy()[ig], om.rgb[n0 + io].astype(np.float32))
    assert np.all(gm.wpos[n0:ng].cpu().numpy() == 1.0)
    assert np.max(np.abs(gm.wrgb[n0:ng].cpu().numpy()[ig] - om.wrgb[n0 + io]), initial=0) <= 1e-5
    return dict(old_points=n0, fragile_points=int(fq.sum()), fragile_pixels=int(fp.sum()),
                appended=len(common), flipped=len(only_g) + len(only_o))


def test_frames_against_oracle(dev):
    h, cam, xyz, rgb = _frame(dev, synth.seed_for(6))
    H, W = xyz.shape[:2]
    gm = st.PointModel(4 * W * H, dev)
    poses = [(np.eye(3, dtype=np.float32), np.zeros(3, np.float32)),
             (_rot_y(0.02), np.array([0.6, -0.2, 0.3], np.float32)),
             (_rot_y(-0.015), np.array([-0.4, 0.1, -0.2], np.float32))]
    xyz_np = xyz.cpu().numpy()
    img_np = rgb.cpu().numpy()
    merged = 0
    for R, t in poses:
        om = _oracle_from(gm)
        n0 = om.count
        st.stereo_mosaic_frame(h, gm, xyz, rgb, cam, R, t, tau=0.8)
        torch.cuda.synchronize()
        dropped, mg = oracle.mosaic_frame(om, xyz_np, img_np, cam.f, cam.cx, cam.cy, R, t, 0.8, margins=MARGINS)
        assert dropped == 0 and int(gm.dropped.item()) == 0
        stats = _compare(gm, om, n0, mg, R, t, cam, W)
        print(f"\nmosaic frame: {stats}")
        assert stats["fragile_points"] <= 0.05 * max(n0, 1)     # the exemption stays small
        merged += int((om.wpos[:n0] >= 2.0).sum())
    # the later frames merged points and appended others
    assert merged > 1000 and om.count > np.isfinite(xyz_np[..., 2]).sum()
    h.close()


def test_capacity_overflow(dev):
    h, cam, xyz, rgb = _frame(dev, synth.seed_for(6, 1), 96, 64)
    cap = 1500
    gm = st.PointModel(cap, dev)
    om = oracle.PointModel(cap)
    I3, Z3 = np.eye(3, dtype=np.float32), np.zeros(3, np.float32)
    st.stereo_mosaic_frame(h, gm, xyz, rgb, cam, I3, Z3, tau=0.5)
    torch.cuda.synchronize()
    dropped, mg = oracle.mosaic_frame(om, xyz.cpu().numpy(), rgb.cpu().numpy(), cam.f, cam.cx, cam.cy, I3, Z3,
                                      0.5, margins=MARGINS)
    assert dropped > 0 and int(gm.dropped.item()) == dropped
    _compare(gm, om, 0, mg, I3, Z3, cam, xyz.shape[1])
    h.close()
