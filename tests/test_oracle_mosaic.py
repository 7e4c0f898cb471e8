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


def test_equal_depth_tie_goes_to_the_smaller_index():
    """Two model points at the same depth on the centre ray: the one with the
    smaller index is kept and merges (hand-derived)."""
    W, H, f, cx, cy = 5, 5, 10.0, 2.0, 2.0
    m = oracle.PointModel(10)
    m.pos[0] = [0.0, 0.0, 10.0]
    m.pos[1] = [0.0, 0.0, 10.0]
    m.wpos[:2] = 1.0
    m.wrgb[:2] = 1.0
    m.count = 2
    xyz = np.full((H, W, 3), np.nan, np.float32)
    xyz[2, 2] = [0.0, 0.0, 10.2]
    img = np.zeros((H, W, 3), np.uint8)
    _, mg = oracle.mosaic_frame(m, xyz, img, f, cx, cy, I3, Z3, 0.5, margins=(1e-3, 1e-6))
    assert m.count == 2 and m.wpos[0] == 2.0 and m.wpos[1] == 1.0
    assert abs(m.pos[0, 2] - (10.0 + float(np.float32(10.2))) / 2) < 1e-12
    # the tie itself is a decision a narrower precision could take differently
    assert mg["fragile_pix"][2, 2] and mg["fragile_pt"].all()


def test_decision_margins():
    """Margins: a point whose projection lies on a rounding edge marks both
    pixels of the edge; a merge test at its threshold marks its pixel;
    decisions far from any edge mark nothing."""
    W, H, f, cx, cy = 8, 6, 10.0, 3.0, 2.0
    m = oracle.PointModel(20)
    # pixel (u, v) = (5, 2): X/Z * f + cx = 5 -> X = 2 Z / f; exactly centred
    m.pos[0] = [2.0, 0.0, 10.0]
    # u + 1/2 = 3.5 + 1/2 = 4: on the edge between pixels 3 and 4 of row 3
    m.pos[1] = [0.5, 1.0, 10.0]
    m.wpos[:2] = 1.0
    m.wrgb[:2] = 1.0
    m.count = 2
    xyz = np.full((H, W, 3), np.nan, np.float32)
    xyz[2, 5] = [2.0, 0.0, 10.5]          # |Q.z - X.z| = 0.5 = tau exactly
    img = np.zeros((H, W, 3), np.uint8)
    _, mg = oracle.mosaic_frame(m, xyz, img, f, cx, cy, I3, Z3, 0.5, margins=(1e-3, 1e-6))
    fp = mg["fragile_pix"]
    assert fp[2, 5]                                        # merge test at its threshold
    assert fp[3, 3] and fp[3, 4]                           # both sides of the rounding edge
    assert fp.sum() == 3
    assert mg["fragile_pt"].tolist() == [True, True]
    assert m.wpos[0] == 2.0                                # |dz| <= tau merges
    # away from the edges nothing is marked
    m2 = oracle.PointModel(20)
    m2.pos[0] = [2.0, 0.0, 10.0]
    m2.wpos[0] = m2.wrgb[0] = 1.0
    m2.count = 1
    xyz[2, 5] = [2.0, 0.0, 10.2]
    _, mg = oracle.mosaic_frame(m2, xyz, img, f, cx, cy, I3, Z3, 0.5, margins=(1e-3, 1e-6))
    assert not mg["fragile_pix"].any() and not mg["fragile_pt"].any()
    assert m2.count == 1 and m2.wpos[0] == 2.0
