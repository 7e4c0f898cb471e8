"""Pins of the oracle's point-based TSDF mosaicking (Sec. II, GPU-based TSDF
mosaicking): the empty model takes every valid pixel; a frame merged into
the model built from itself maps every point back onto its own pixel
(weights double, positions and colours stay); a camera translated by a
whole number of pixels over a fronto-parallel plane merges the overlap and
appends exactly the newly seen strip; the z-buffer keeps the nearer point;
the truncation band and the capacity limit; the colour weight's extremes."""
import numpy as np

import oracle


def _plane_frame(W, H, f, Z0, cx, cy, rgb_seed=0):
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    xyz = np.stack([(u - cx) * Z0 / f, (v - cy) * Z0 / f, np.full_like(u, Z0)], -1).astype(np.float32)
    img = np.random.default_rng(rgb_seed).integers(0, 256, (H, W, 3), dtype=np.uint8)
    return xyz, img


I3 = np.eye(3, dtype=np.float32)
Z3 = np.zeros(3, np.float32)


def test_empty_model_appends_valid_pixels_in_order():
    W, H, f = 7, 5, 50.0
    xyz, img = _plane_frame(W, H, f, 10.0, 3.0, 2.0)
    xyz[1, 2] = np.nan
    m = oracle.PointModel(100)
    assert oracle.mosaic_frame(m, xyz, img, f, 3.0, 2.0, I3, Z3, 0.5) == 0
    keep = ~np.isnan(xyz[..., 2])
    assert m.count == keep.sum()
    assert np.allclose(m.pos[:m.count], xyz[keep].astype(np.float64))
    assert np.array_equal(m.rgb[:m.count], img[keep].astype(np.float64))
    assert np.all(m.wpos[:m.count] == 1.0)
    # colour weight: 1 at the image centre, decreasing towards the corners
    rank = np.cumsum(keep.ravel()) - 1
    assert m.wrgb[rank[np.ravel_multi_index((2, 3), (H, W))]] == 1.0
    assert 0.1 <= m.wrgb[rank[0]] < m.wrgb[rank[np.ravel_multi_index((1, 1), (H, W))]] <= 1.0


def test_frame_merged_into_its_own_model():
    W, H, f, cx, cy = 40, 30, 60.0, 19.5, 14.5
    xyz, img = _plane_frame(W, H, f, 25.0, cx, cy)
    m = oracle.PointModel(5000)
    oracle.mosaic_frame(m, xyz, img, f, cx, cy, I3, Z3, 0.5)
    n = m.count
    pos0, rgb0, c0 = m.pos[:n].copy(), m.rgb[:n].copy(), m.wrgb[:n].copy()
    oracle.mosaic_frame(m, xyz, img, f, cx, cy, I3, Z3, 0.5)
    assert m.count == n                                       # every pixel found its own point
    assert np.allclose(m.pos[:n], pos0, atol=1e-12)
    assert np.allclose(m.rgb[:n], rgb0, atol=1e-9)
    assert np.all(m.wpos[:n] == 2.0)
    assert np.allclose(m.wrgb[:n], 2 * c0)


def test_translated_camera_merges_overlap_and_appends_new_strip():
    """Camera moved right by k pixels' worth over a plane at depth Z0: pixel
    (u, v) of the new frame sees the point of pixel (u + k, v) of the first."""
    W, H, f, cx, cy, Z0, k = 32, 16, 40.0, 15.5, 7.5, 20.0, 5
    xyz, img = _plane_frame(W, H, f, Z0, cx, cy)
    m = oracle.PointModel(10000)
    oracle.mosaic_frame(m, xyz, img, f, cx, cy, I3, Z3, 0.25)
    n = m.count
    tx = k * Z0 / f                                           # camera centre at (tx, 0, 0)
    t = np.array([-tx, 0.0, 0.0], np.float32)                 # X_cam = P - (tx, 0, 0)
    xyz_b = xyz.copy()                                        # same camera-frame geometry
    img_b = np.random.default_rng(5).integers(0, 256, (H, W, 3), dtype=np.uint8)
    oracle.mosaic_frame(m, xyz_b, img_b, f, cx, cy, I3, t, 0.25)
    assert m.count == n + k * H                               # the strip u >= W - k is new
    merged = m.wpos[:n] == 2.0
    assert merged.sum() == (W - k) * H
    # merged points: first-frame columns u >= k; positions unchanged (same world point)
    cols = np.tile(np.arange(W), H)
    assert np.array_equal(merged, cols >= k)
    new = m.pos[n:m.count]
    assert np.allclose(new[:, 0], (np.tile(np.arange(W - k, W), H) - cx) * Z0 / f + tx, atol=1e-4)


def test_zbuffer_keeps_the_nearer_point_and_truncation():
    W, H, f, cx, cy = 5, 5, 10.0, 2.0, 2.0
    m = oracle.PointModel(50)
    # two model points on the centre ray: the farther one first (index 0)
    m.pos[0] = [0.0, 0.0, 20.0]
    m.pos[1] = [0.0, 0.0, 10.0]
    m.wpos[:2] = 1.0
    m.wrgb[:2] = 1.0
    m.count = 2
    xyz = np.full((H, W, 3), np.nan, np.float32)
    img = np.zeros((H, W, 3), np.uint8)
    xyz[2, 2] = [0.0, 0.0, 10.4]
    oracle.mosaic_frame(m, xyz, img, f, cx, cy, I3, Z3, 0.5)
    assert m.count == 2 and m.wpos[1] == 2.0 and m.wpos[0] == 1.0
    assert abs(m.pos[1, 2] - 10.2) < 1e-6
    xyz[2, 2] = [0.0, 0.0, 12.0]                              # outside the band: a new point
    oracle.mosaic_frame(m, xyz, img, f, cx, cy, I3, Z3, 0.5)
    assert m.count == 3 and m.wpos[1] == 2.0 and abs(m.pos[2, 2] - 12.0) < 1e-6


def test_capacity_limit_drops_appends():
    W, H, f = 6, 4, 30.0
    xyz, img = _plane_frame(W, H, f, 5.0, 2.5, 1.5)
    m = oracle.PointModel(10)
    assert oracle.mosaic_frame(m, xyz, img, f, 2.5, 1.5, I3, Z3, 0.5) == W * H - 10
    assert m.count == 10
    assert np.allclose(m.pos[:10], xyz.reshape(-1, 3)[:10])
