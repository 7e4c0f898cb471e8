"""Pins for the oracle's left-right check, outlier removal and hole filling
(Sec. II-B) and for the gray conversion.  Expected values are derived by hand
from small maps whose answer can be counted."""
import numpy as np
import pytest

import oracle

INV = oracle.INVALID


def test_gray_fixed_point():
    v = np.arange(256, dtype=np.uint8)
    rgb = np.stack([v, v, v], -1)[None]
    assert np.array_equal(oracle.gray(rgb)[0], v)   # weights sum to 256
    rgb = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255], [10, 20, 30]]], np.uint8)
    assert oracle.gray(rgb)[0].tolist() == [77, 149, 29, 18]


def test_lr_check_hand():
    dL = np.array([[INV, 1, 2, 2, 3, 0, 5, 1]], np.int16)
    dR = np.array([[0, 1, 3, INV, 9, 0, 3, 2]], np.int16)
    # x=1: u=0, dR=0, |1-0|=1 keep;  x=2: u=0, |2-0|=2 drop;  x=3: u=1, |2-1| keep
    # x=4: u=1, |3-1|=2 drop;        x=5: u=5, |0-0| keep;   x=6: u=1, |5-1| drop
    # x=7: u=6, |1-3|=2 drop
    out = oracle.lr_check(dL, dR, 1)
    assert out.tolist() == [[INV, 1, INV, 2, INV, 0, INV, INV]]
    out0 = oracle.lr_check(dL, dR, 0)
    assert out0.tolist() == [[INV, INV, INV, INV, INV, 0, INV, INV]]
    # correspondence outside the image
    dL2 = np.array([[0, 3, INV]], np.int16)
    dR2 = np.array([[3, 0, 0]], np.int16)
    assert oracle.lr_check(dL2, dR2, 1).tolist() == [[INV, INV, INV]]


def test_outlier_spike_removed_rest_kept():
    o = np.full((25, 25), 10, np.int16)
    o[12, 12] = 20
    out = oracle.outlier_removal(o, 10, 2.5)
    want = o.copy()
    want[12, 12] = INV
    assert np.array_equal(out, want)


def test_outlier_radius_must_fit_in_image():
    o = np.full((5, 5), 3, np.int16)
    assert np.all(oracle.outlier_removal(o, 10, 2.5) == INV)
    # with r = 4 only pixels on the image border have 4 steps in some direction
    want = np.full((5, 5), 3, np.int16)
    want[1:4, 1:4] = INV
    assert np.array_equal(oracle.outlier_removal(o, 4, 2.5), want)
    assert np.all(oracle.outlier_removal(o, 2, 2.5) == 3)
    row = np.full((1, 11), 3, np.int16)
    out = oracle.outlier_removal(row, 10, 2.5)
    want = np.full((1, 11), INV, np.int16)
    want[0, 0] = want[0, 10] = 3          # only the ends see 10 steps
    assert np.array_equal(out, want)


def test_outlier_threshold_is_strict():
    row = (2 * np.arange(30)).astype(np.int16)[None]      # slope 2
    assert np.all(oracle.outlier_removal(row, 10, 2.5) == row)
    assert np.all(oracle.outlier_removal(row, 10, 2.0) == INV)   # 2 < 2 is false
    yy, xx = np.mgrid[0:30, 0:30]
    ramp = (3 * xx).astype(np.int16)                          # rows constant
    assert np.array_equal(oracle.outlier_removal(ramp, 10, 2.5), ramp)
    diag = (3 * xx + 3 * yy).astype(np.int16)                 # anti-diagonal constant
    # only the anti-diagonal directions are smooth; a pixel keeps its value
    # when 10 anti-diagonal steps fit in the 30x30 image one way or the other
    room = ((xx + 10 <= 29) & (yy - 10 >= 0)) | ((xx - 10 >= 0) & (yy + 10 <= 29))
    assert np.array_equal(oracle.outlier_removal(diag, 10, 2.5), np.where(room, diag, INV))
    steep = (3 * xx + 6 * yy).astype(np.int16)                # no smooth direction
    assert np.all(oracle.outlier_removal(steep, 1, 2.5) == INV)


def test_outlier_invalid_pixels_block_directions():
    o = np.full((21, 21), 5, np.int16)
    o[10, :] = INV          # a hole row
    o[:, 10] = INV          # and a hole column: four 10x10 quadrants remain
    q = np.arange(21) % 11  # position inside a quadrant (10 on the cross)
    qy, qx = np.meshgrid(q, q, indexing="ij")
    # 9 steps fit inside a quadrant only from its edge rows/columns
    edge = (qx == 0) | (qx == 9) | (qy == 0) | (qy == 9)
    want = np.where((o != INV) & edge, 5, INV).astype(np.int16)
    assert np.array_equal(oracle.outlier_removal(o, 9, 2.5), want)
    # 10 steps never fit inside a 10-pixel quadrant
    assert np.all(oracle.outlier_removal(o, 10, 2.5) == INV)


def _plus_map(values):
    o = np.full((11, 11), INV, np.int16)
    (r, vr), (l, vl), (u, vu), (d, vd) = values
    o[5, 5 + r] = vr
    o[5, 5 - l] = vl
    o[5 - u, 5] = vu
    o[5 + d, 5] = vd
    return o


def test_fill_radial_weighted_mean():
    o = _plus_map([(2, 10), (3, 20), (1, 30), (4, 14)])
    # weights 51-s: 49, 48, 50, 47; sum 194; weighted sum 3608; 3608/194 = 18.6
    assert oracle.fill_radial(o, 50, 4)[5, 5] == 19
    assert oracle.fill_radial(o, 50, 5)[5, 5] == INV
    # halves round up (toward +inf)
    assert oracle.fill_radial(_plus_map([(1, 1), (1, 1), (1, 2), (1, 2)]), 50, 4)[5, 5] == 2
    assert oracle.fill_radial(_plus_map([(1, -1), (1, -1), (1, -2), (1, -2)]), 50, 4)[5, 5] == -1
    # a value beyond the radius is not found
    assert oracle.fill_radial(_plus_map([(2, 10), (3, 20), (1, 30), (4, 14)]), 3, 4)[5, 5] == INV
    # valid pixels are untouched
    f = oracle.fill_radial(o, 50, 4)
    assert f[5, 7] == 10 and f[5, 2] == 20


def test_disc_area_gauss_circle():
    # number of lattice points with x^2 + y^2 <= r^2 (Gauss circle problem)
    assert [oracle.disc_area(r) for r in (0, 1, 2, 3, 4, 5, 10, 20)] == [1, 5, 13, 29, 49, 81, 317, 1257]


def test_fill_disc():
    o = np.full((41, 41), 7, np.int16)
    o[20, 20] = INV
    assert oracle.fill_disc(o, 20)[20, 20] == 7
    # corner hole: 335 lattice points of the quarter disc lie in the image,
    # minus the hole itself = 334 >= 315
    c = np.full((41, 41), 7, np.int16)
    c[0, 0] = INV
    assert oracle.fill_disc(c, 20)[0, 0] == 7
    assert oracle.fill_disc(c, 20, 335)[0, 0] == INV
    assert oracle.fill_disc(c, 20, 334)[0, 0] == 7
    # mean 10.5 rounds up
    # the 1256 disc pixels around the centre: 608 with dx > 0 (value 11), 608
    # with dx < 0 (value 10), 20 above (10) and 20 below (11) on dx = 0
    h = np.full((41, 41), 10, np.int16)
    h[:, 21:] = 11
    h[21:, 20] = 11
    h[20, 20] = INV
    assert oracle.fill_disc(h, 20)[20, 20] == 11
    # a sparse field (one valid pixel in 5) is not filled
    s = np.full((41, 41), INV, np.int16)
    s[::5, :] = 3
    assert oracle.fill_disc(s, 20)[20, 20] == 3          # on a valid row: untouched
    s2 = np.full((41, 41), INV, np.int16)
    s2[1::5, :] = 3                                       # ~ 1257/5 valid in the disc
    assert oracle.fill_disc(s2, 20)[20, 20] == INV


def test_postprocess_round_schedule():
    """A 15x15 plateau (value 50) on a zero background: with r = 10 the plateau
    centre is removed and refilled with 50, so one round changes nothing; with
    r = 20 no plateau pixel has 20 smooth steps, the whole plateau becomes a
    hole and is filled from the zero background."""
    o = np.zeros((64, 64), np.int16)
    o[25:40, 25:40] = 50
    p1 = oracle.Params(outlier_rounds=1)
    assert np.array_equal(oracle.postprocess(o, p1), o)
    after_first_outlier = oracle.outlier_removal(o, 10, 2.5)
    assert np.all(after_first_outlier[30:35, 30:35] == INV)
    assert np.sum(after_first_outlier == INV) == 25
    p2 = oracle.Params(outlier_rounds=2)
    assert np.all(oracle.postprocess(o, p2) == 0)
    p3 = oracle.Params(outlier_rounds=3)
    assert np.all(oracle.postprocess(o, p3) == 0)
    # with a constant radius (dr = 0) the second round changes nothing either
    p2c = oracle.Params(outlier_rounds=2, dr=0)
    assert np.array_equal(oracle.postprocess(o, p2c), o)


def test_postprocess_spike_block():
    o = np.full((64, 64), 10, np.int16)
    o[29:32, 29:32] = 40
    assert np.all(oracle.postprocess(o, oracle.Params()) == 10)
