"""Pins for the oracle's ZNCC, winner-take-all and sub-pixel steps (Sec. II-A).

None of these re-type the oracle's formula: they compare it with numpy's
Pearson correlation (a library routine), with exact recovery on synthetic
shifts, with brute-force argmax over library correlations, with closed forms
and with invariants (bounds, affine invariance, mirror symmetry).
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(1234)


def _window(img, x, y, r, sampling=0):
    w = img[y - r:y + r + 1, x - r:x + r + 1].astype(np.float64)
    if sampling == oracle.SAMPLE_CHESSBOARD:
        dy, dx = np.mgrid[-r:r + 1, -r:r + 1]
        w = w[(dx + dy) % 2 == 0]
    return w.ravel()


@pytest.mark.parametrize("sampling", [oracle.SAMPLE_FULL, oracle.SAMPLE_CHESSBOARD])
@pytest.mark.parametrize("r", [1, 2, 5, 7])
def test_zncc_equals_pearson_correlation(r, sampling):
    H, W = 30, 40
    L = RNG.integers(0, 256, (H, W), dtype=np.uint8)
    R = RNG.integers(0, 256, (H, W), dtype=np.uint8)
    for _ in range(40):
        y = int(RNG.integers(r, H - r))
        x = int(RNG.integers(r, W - r))
        d = int(RNG.integers(0, x - r + 1))
        want = np.corrcoef(_window(L, x, y, r, sampling), _window(R, x - d, y, r, sampling))[0, 1]
        got = oracle.zncc(L, R, r, x, y, d, sampling)
        assert abs(got - want) <= 1e-13, (x, y, d, got, want)


def test_invalid_candidates_are_nan_and_bounds():
    H, W, r = 12, 9, 2
    L = RNG.integers(0, 256, (H, W), dtype=np.uint8)
    R = RNG.integers(0, 256, (H, W), dtype=np.uint8)
    for y in range(H):
        for x in range(W):
            for d in range(-3, 8):
                inside = (r <= y < H - r) and (r <= x < W - r) and (r <= x - d < W - r)
                assert oracle.candidate_valid(W, H, r, x, y, d) == inside
                v = oracle.zncc(L, R, r, x, y, d)
                if inside:
                    assert -1.0 - 1e-12 <= v <= 1.0 + 1e-12
                else:
                    assert np.isnan(v)


def test_affine_invariance_and_role_swap():
    H, W, r = 20, 30, 3
    L = RNG.integers(0, 127, (H, W), dtype=np.uint8)
    R = RNG.integers(0, 256, (H, W), dtype=np.uint8)
    L2 = (2 * L.astype(np.int32) + 3).astype(np.uint8)      # exact in u8
    for (x, y, d) in [(10, 8, 2), (20, 10, 7), (26, 16, 0), (15, 5, 12)]:
        a = oracle.zncc(L, R, r, x, y, d)
        b = oracle.zncc(L2, R, r, x, y, d)
        assert abs(a - b) < 1e-13
        # swapping the images and mirroring the disparity gives the same value
        c = oracle.zncc(R, L, r, x - d, y, -d)
        assert abs(a - c) < 1e-13


def test_constant_window_is_zero():
    H, W, r = 15, 15, 2
    L = np.full((H, W), 77, np.uint8)
    R = RNG.integers(0, 256, (H, W), dtype=np.uint8)
    assert oracle.zncc(L, R, r, 7, 7, 1) == 0.0
    assert oracle.zncc(R, L, r, 7, 7, 1) == 0.0


def _textured(H, W, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, (H, W), dtype=np.uint8)


@pytest.mark.parametrize("dstar", [0, 3, 9])
def test_exact_recovery_constant_shift(dstar):
    """R(x) = L(x + d*): rho(d*) = 1 and the WTA returns d* on every pixel whose
    true candidate is valid."""
    H, W, r, D = 20, 48, 3, 14
    big = _textured(H, W + dstar, 7)
    L = big[:, :W].copy()
    R = big[:, dstar:dstar + W].copy()     # R(u) = L(u + d*)
    m = oracle.match(L, R, 0, D, r)
    for y in range(r, H - r):
        for x in range(r + dstar, W - r):
            assert abs(oracle.zncc(L, R, r, x, y, dstar) - 1.0) < 1e-12
            assert m["dL"][y, x] == dstar
            assert abs(m["sub"][y, x] - dstar) <= 0.5
    # right view: u's best left match is u + d* whenever that is valid
    for y in range(r, H - r):
        for u in range(r, W - r - dstar):
            assert m["dR"][y, u] == dstar


def test_exact_recovery_piecewise_shift():
    """Two vertical bands with different integer shifts; pixels whose window
    does not straddle the seam recover their band's shift exactly."""
    H, W, r, D = 18, 64, 2, 12
    src = _textured(H, W + 20, 11)
    L = src[:, :W].copy()
    R = np.zeros_like(L)
    shift = np.where(np.arange(W) < 32, 4, 9)
    for u in range(W):
        R[:, u] = src[:, u + shift[u]]
    m = oracle.match(L, R, 0, D, r)
    for y in range(r, H - r):
        for x in range(W):
            d = 4 if x - 4 < 32 else 9
            u = x - d
            if not (r <= u < W - r and r <= x < W - r):
                continue
            if any(shift[u + k] != d for k in range(-r, r + 1) if 0 <= u + k < W):
                continue
            assert m["dL"][y, x] == d, (x, y)


def test_brute_force_argmax_tiny():
    """On tiny images, the WTA maps equal an argmax over library correlations."""
    for sampling in (oracle.SAMPLE_FULL, oracle.SAMPLE_CHESSBOARD):
        H, W, r, dmin, D = 9, 14, 1, -2, 6
        L = _textured(H, W, 21)
        R = _textured(H, W, 22)
        m = oracle.match(L, R, dmin, D, r, sampling)
        for y in range(H):
            for x in range(W):
                rho = []
                for k in range(D):
                    d = dmin + k
                    if r <= y < H - r and r <= x < W - r and r <= x - d < W - r:
                        rho.append(np.corrcoef(_window(L, x, y, r, sampling),
                                               _window(R, x - d, y, r, sampling))[0, 1])
                    else:
                        rho.append(-np.inf)
                rho = np.array(rho)
                if np.all(np.isinf(rho)):
                    assert m["dL"][y, x] == oracle.INVALID
                else:
                    assert m["dL"][y, x] == dmin + int(np.argmax(rho))   # first max
                # right pixel u = x: best over d of rho(u + d, d)
                rr = []
                for k in range(D):
                    d = dmin + k
                    xl = x + d
                    if r <= y < H - r and r <= xl < W - r and r <= x < W - r:
                        rr.append(np.corrcoef(_window(L, xl, y, r, sampling),
                                              _window(R, x, y, r, sampling))[0, 1])
                    else:
                        rr.append(-np.inf)
                rr = np.array(rr)
                if np.all(np.isinf(rr)):
                    assert m["dR"][y, x] == oracle.INVALID
                else:
                    assert m["dR"][y, x] == dmin + int(np.argmax(rr))


def test_mirror_symmetry():
    """With L' = flip(R) and R' = flip(L), the left map of the mirrored pair is
    the mirrored right map of the original pair (ties included)."""
    H, W, r, D = 16, 40, 2, 10
    L = _textured(H, W, 31)
    R = _textured(H, W, 32)
    m = oracle.match(L, R, 0, D, r)
    mm = oracle.match(R[:, ::-1], L[:, ::-1], 0, D, r)
    near_tie = (mm["gapL"] < 1e-12) | (m["gapR"][:, ::-1] < 1e-12)
    assert np.array_equal(np.where(near_tie, 0, mm["dL"]),
                          np.where(near_tie, 0, m["dR"][:, ::-1]))


def test_range_bounds():
    H, W, r, dmin, D = 20, 50, 2, -4, 9
    L = _textured(H, W, 41)
    R = _textured(H, W, 42)
    m = oracle.match(L, R, dmin, D, r)
    for key in ("dL", "dR"):
        v = m[key]
        ok = (v == oracle.INVALID) | ((v >= dmin) & (v < dmin + D))
        assert ok.all()
    sub = m["sub"]
    valid = m["dL"] != oracle.INVALID
    assert np.all(np.abs(sub[valid] - m["dL"][valid]) <= 0.5)
    assert np.all(np.isnan(sub[~valid]))


def test_parabola_closed_form():
    for d0 in [-0.49, -0.3, 0.0, 0.17, 0.4999]:
        for a in [0.01, 1.0, 7.5]:
            b = 0.2
            c = [a * (t - d0) ** 2 + b for t in (-1.0, 0.0, 1.0)]
            assert abs(oracle.parabola(*c) - d0) < 1e-12
    assert oracle.parabola(0.5, 0.5, 0.5) == 0.0        # flat: no curvature
    assert oracle.parabola(0.2, 0.5, 0.2) == 0.0        # a maximum, not a minimum
    assert oracle.parabola(0.0, 0.0, 10.0) == -0.5      # clamped
    assert oracle.parabola(10.0, 0.0, 0.0) == 0.5


def test_subpixel_skipped_at_range_edges():
    """The parabola needs both neighbours: at the first/last candidate the
    sub-pixel value is the integer winner itself."""
    H, W, r = 12, 40, 2
    big = _textured(H, W + 6, 51)
    L = big[:, :W].copy()
    R = big[:, 6:6 + W].copy()            # true shift 6
    d, gap, sub = oracle.wta_left_pixel(L, R, 6, 5, r, 20, 6)  # range 6..10, 6 at the edge
    assert d == 6 and sub == 6.0
    d, gap, sub = oracle.wta_left_pixel(L, R, 2, 5, r, 20, 6)  # range 2..6, 6 at the edge
    assert d == 6 and sub == 6.0
