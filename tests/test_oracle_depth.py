"""Pins of the oracle's disparity -> points / normals step (Sec. II:
physical depth from disparity after calibration, the reprojection of a
rectified pair), against closed forms: a hand-computed pixel, an exact plane
(every point on it, every normal equal to its normal), a sphere (normals
radial up to the central-difference error), and the missing-data rules."""
import numpy as np

import oracle


def test_single_pixel_by_hand():
    d = np.full((3, 3), np.nan)
    d[1, 1] = 25.0
    f, cx, cy, B = 500.0, 0.0, 2.0, 5.0            # pixel (u, v) = (1, 1)
    xyz, nrm = oracle.depth_points(d, f, cx, cy, B)
    Z = 500.0 * 5.0 / 25.0                          # 100
    assert np.allclose(xyz[1, 1], [(1 - 0.0) * Z / f, (1 - 2.0) * Z / f, Z], rtol=0, atol=1e-12)
    assert np.isnan(xyz[0, 0]).all() and np.isnan(nrm).all()


def test_principal_point_offset_shifts_disparity():
    d = np.full((1, 1), 20.0)
    a, _ = oracle.depth_points(d, 400.0, 0.0, 0.0, 3.0, doffs=5.0)
    assert abs(a[0, 0, 2] - 400.0 * 3.0 / 25.0) < 1e-12
    b, _ = oracle.depth_points(d, 400.0, 0.0, 0.0, 3.0, doffs=-20.0)   # d + doffs = 0: undefined
    assert np.isnan(b).all()


def _plane_disparity(n, h, W, H, f, cx, cy, B, doffs):
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    ray = np.stack([(u - cx) / f, (v - cy) / f, np.ones_like(u)], -1)
    Z = h / (ray @ n)                               # n . (Z ray) = h
    return f * B / Z - doffs, Z


def test_plane_points_and_normals_exact():
    W, H, f, cx, cy, B, doffs = 40, 30, 300.0, 19.5, 14.0, 4.0, 2.5
    n = np.array([0.2, -0.3, -1.0])
    n /= np.linalg.norm(n)                          # faces the camera (n_z < 0)
    h = n @ np.array([0.0, 0.0, 80.0])
    d, Z = _plane_disparity(n, h, W, H, f, cx, cy, B, doffs)
    xyz, nrm = oracle.depth_points(d, f, cx, cy, B, doffs)
    assert np.allclose(xyz[..., 2], Z, rtol=1e-12)
    assert np.max(np.abs(xyz @ n - h)) < 1e-9 * abs(h)
    inner = nrm[1:-1, 1:-1].reshape(-1, 3)
    assert np.max(np.abs(inner - n)) < 1e-9
    assert np.isnan(nrm[0]).all() and np.isnan(nrm[-1]).all()
    assert np.isnan(nrm[:, 0]).all() and np.isnan(nrm[:, -1]).all()


def test_normals_face_the_camera_and_are_unit():
    """A plane seen from behind its stated normal still gets the normal that
    faces the camera."""
    W, H, f, cx, cy, B = 20, 20, 200.0, 10.0, 10.0, 2.0
    n = np.array([0.1, 0.1, 1.0])
    n /= np.linalg.norm(n)                          # points away from the camera
    d, Z = _plane_disparity(n, n @ np.array([0.0, 0.0, 50.0]), W, H, f, cx, cy, B, 0.0)
    _, nrm = oracle.depth_points(d, f, cx, cy, B)
    inner = nrm[1:-1, 1:-1].reshape(-1, 3)
    assert np.max(np.abs(inner + n)) < 1e-9
    assert np.allclose(np.linalg.norm(inner, axis=1), 1.0, atol=1e-12)


def test_sphere_normals_radial():
    """Central differences on a sphere of radius 40 at distance 100: normals
    within 1e-3 of the radial direction (second-order error of the
    differences)."""
    W, H, f, cx, cy, B = 64, 64, 400.0, 31.5, 31.5, 3.0
    c = np.array([0.0, 0.0, 100.0])
    rad = 40.0
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    ray = np.stack([(u - cx) / f, (v - cy) / f, np.ones_like(u)], -1)
    # nearest intersection of Z * ray with the sphere
    a = np.sum(ray * ray, -1)
    bq = -2.0 * ray @ c
    cq = c @ c - rad * rad
    Z = (-bq - np.sqrt(bq * bq - 4 * a * cq)) / (2 * a)
    d = f * B / Z
    xyz, nrm = oracle.depth_points(d, f, cx, cy, B)
    radial = (xyz - c) / rad
    err = np.linalg.norm(nrm[2:-2, 2:-2] - radial[2:-2, 2:-2], axis=-1)
    assert np.max(err) < 1e-3


def test_missing_neighbour_invalidates_normal():
    d = np.full((5, 5), 10.0)
    d[2, 3] = np.nan
    xyz, nrm = oracle.depth_points(d, 100.0, 2.0, 2.0, 1.0)
    assert np.isnan(xyz[2, 3]).all() and not np.isnan(xyz[2, 2]).any()
    assert np.isnan(nrm[2, 2]).all()                # right neighbour missing
    assert not np.isnan(nrm[1, 1]).any()
