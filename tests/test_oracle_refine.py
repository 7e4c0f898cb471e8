"""Pins for the oracle's improved Laplacian refinement (Sec. II-C, Eqs. 1-4):
a hand-derived worked example (tests/golden/laplacian_3px.txt), identities
(K = 0, constant maps, interior of a linear ramp) and the o-update's limits
(eta -> infinity keeps the nearest integer; eta = 0 follows the ZNCC)."""
import os

import numpy as np
import pytest

import oracle

INV = oracle.INVALID
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _flat_cost(H, W, D, rho=0.5):
    return np.full((H, W, D), 1.0 - rho)


def test_worked_example_golden():
    rows = np.loadtxt(os.path.join(GOLDEN, "laplacian_3px.txt"))
    o = np.array([[0, 3, 6]], np.int16)
    for K, d0, d1, d2, o0, o1, o2 in rows:
        p = oracle.Params(d_min=0, num_disp=16, smooth_radius=1, smooth_iters=int(K),
                          alpha=0.1, eta=1.0)
        d, on = oracle.refine(o, cost=_flat_cost(1, 3, 16), p=p)
        assert np.allclose(d[0], [d0, d1, d2], atol=1e-12, rtol=0)
        assert on[0].tolist() == [o0, o1, o2]


def test_zero_iterations_is_identity():
    rng = np.random.default_rng(3)
    o = rng.integers(0, 30, (20, 25)).astype(np.int16)
    o[rng.random((20, 25)) < 0.2] = INV
    p = oracle.Params(num_disp=32, smooth_radius=2, smooth_iters=0)
    d, on = oracle.refine(o, cost=_flat_cost(20, 25, 32), p=p)
    v = o != INV
    assert np.array_equal(d[v], o[v].astype(float))
    assert np.all(np.isnan(d[~v]))
    assert np.array_equal(on, o)


def test_constant_map_is_fixed_point():
    o = np.full((17, 23), 12, np.int16)
    o[5:8, 5:9] = INV
    p = oracle.Params(num_disp=32, smooth_radius=3, smooth_iters=4)
    d, on = oracle.refine(o, cost=_flat_cost(17, 23, 32), p=p)
    v = o != INV
    assert np.all(d[v] == 12.0)
    assert np.array_equal(on, o)


def test_linear_ramp_interior_preserved():
    """The improved (non-shrinking) Laplacian leaves a linear ramp unchanged
    wherever the whole box lies inside the map."""
    H, W, rs = 30, 40, 3
    yy, xx = np.mgrid[0:H, 0:W]
    o = (xx // 1 + 10).astype(np.int16)
    p = oracle.Params(num_disp=64, smooth_radius=rs, smooth_iters=3, eta=1e6)
    d, on = oracle.refine(o, cost=_flat_cost(H, W, 64), p=p)
    K = 3
    m = 2 * rs * K   # influence of the border reaches rs per box mean
    inner = (slice(m, H - m), slice(m, W - m))
    assert np.allclose(d[inner], o[inner], atol=1e-12, rtol=0)


def test_large_eta_keeps_nearest_integer():
    rng = np.random.default_rng(5)
    o = rng.integers(5, 25, (12, 15)).astype(np.int16)
    p = oracle.Params(num_disp=40, smooth_radius=1, smooth_iters=1, eta=1e9)
    d, on = oracle.refine(o, cost=_flat_cost(12, 15, 40, 0.3), p=p)
    nearest = np.floor(d + 0.5)                 # ties (x.5) go to the lower o*
    tie = np.isclose(d - np.floor(d), 0.5)
    nearest[tie] = np.floor(d[tie])
    assert np.array_equal(on, nearest.astype(np.int16))


def test_o_update_follows_zncc_and_skips_nonpositive():
    # a single pixel: dt = o, b = 0, d = o = 7; search [2, 12]
    o = np.array([[7]], np.int16)
    cost = np.full((1, 1, 20), 0.5)            # rho = 0.5: 1/rho = 2
    cost[0, 0, 10] = 1.0 - 0.9                 # rho = 0.9 at d = 10
    p = oracle.Params(num_disp=20, smooth_radius=1, smooth_iters=1, eta=0.01)
    _, on = oracle.refine(o, cost=cost, p=p)
    assert on[0, 0] == 10                      # 1/0.9 + 0.09 < 2
    p = oracle.Params(num_disp=20, smooth_radius=1, smooth_iters=1, eta=0.2)
    _, on = oracle.refine(o, cost=cost, p=p)
    assert on[0, 0] == 7                       # 1/0.9 + 1.8 > 2
    # non-positive ZNCC is never chosen; with no usable candidate o stays
    cost = np.full((1, 1, 20), 1.0)            # rho = 0 everywhere
    cost[0, 0, 3] = 1.0 - 0.1                  # rho = 0.1 only at d = 3
    p = oracle.Params(num_disp=20, smooth_radius=1, smooth_iters=1, eta=0.01)
    _, on = oracle.refine(o, cost=cost, p=p)
    assert on[0, 0] == 3
    cost = np.full((1, 1, 20), 1.5)            # rho = -0.5
    _, on = oracle.refine(o, cost=cost, p=p)
    assert on[0, 0] == 7
    cost = np.full((1, 1, 20), np.nan)         # no valid candidate
    _, on = oracle.refine(o, cost=cost, p=p)
    assert on[0, 0] == 7


def test_cost_volume_and_on_the_fly_zncc_agree():
    rng = np.random.default_rng(9)
    H, W, D, r = 18, 30, 8, 2
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    o = rng.integers(0, D, (H, W)).astype(np.int16)
    p = oracle.Params(num_disp=D, win_radius=r, smooth_radius=2, smooth_iters=2)
    cv = oracle.cost_volume(L, R, 0, D, r)
    d1, o1 = oracle.refine(o, cost=cv, p=p)
    d2, o2 = oracle.refine(o, L=L, R=R, p=p)
    assert np.array_equal(o1, o2)
    assert np.allclose(d1, d2, equal_nan=True, atol=1e-12)
