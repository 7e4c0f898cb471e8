"""Pins for the oracle's soft-argmin variant and its analytic gradient:
central finite differences in FP64, the two temperature limits (tau -> 0 is
the winner-take-all, tau -> infinity the plain mean of the valid
candidates), and the L1 loss by hand."""
import numpy as np
import pytest

import oracle


def _pair(H, W, seed, shift=4):
    rng = np.random.default_rng(seed)
    big = rng.integers(20, 236, (H, W + shift)).astype(np.float64)
    L = big[:, :W].copy()
    R = big[:, shift:shift + W].copy() + rng.normal(0, 6.0, (H, W))
    return L, R


@pytest.mark.parametrize("sampling", [oracle.SAMPLE_FULL, oracle.SAMPLE_CHESSBOARD])
def test_gradient_matches_central_differences(sampling):
    H, W, D, r, tau, h = 20, 26, 8, 2, 0.1, 1e-3
    L, R = _pair(H, W, 17)
    rng = np.random.default_rng(18)
    g = rng.normal(0, 1, (H, W))
    ds, _, hv = oracle.softargmin_fwd(L, R, 0, D, r, tau, sampling)
    g[~hv] = 0.0
    gL, gR = oracle.softargmin_bwd(L, R, 0, D, r, tau, g, sampling)

    def J(Lx, Rx):
        d, _, v = oracle.softargmin_fwd(Lx, Rx, 0, D, r, tau, sampling)
        return float(np.sum(np.where(v, g * d, 0.0)))

    pts = [(int(rng.integers(0, H)), int(rng.integers(0, W))) for _ in range(25)]
    pts += [(10, 12), (5, 20), (r, r + 3)]
    for (y, x) in pts:
        for which, grad in (("L", gL), ("R", gR)):
            Lp, Lm, Rp, Rm = L.copy(), L.copy(), R.copy(), R.copy()
            if which == "L":
                Lp[y, x] += h; Lm[y, x] -= h
            else:
                Rp[y, x] += h; Rm[y, x] -= h
            fd = (J(Lp, Rp) - J(Lm, Rm)) / (2 * h)
            scale = max(1e-3, np.abs(grad).max())
            assert abs(fd - grad[y, x]) <= 1e-6 * scale, (which, y, x, fd, grad[y, x])


def test_small_tau_gives_wta_and_large_tau_the_mean():
    H, W, D, r = 16, 30, 6, 2
    L, R = _pair(H, W, 23, shift=3)
    Lu = np.clip(np.rint(L), 0, 255).astype(np.uint8)
    Ru = np.clip(np.rint(R), 0, 255).astype(np.uint8)
    m = oracle.match(Lu, Ru, 0, D, r)
    ds, lse, hv = oracle.softargmin_fwd(Lu.astype(float), Ru.astype(float), 0, D, r, 1e-4)
    clear = hv & (m["gapL"] > 0.05)
    assert np.allclose(ds[clear], m["dL"][clear], atol=1e-9)
    ds, lse, hv = oracle.softargmin_fwd(Lu.astype(float), Ru.astype(float), 0, D, r, 1e9)
    for y in range(H):
        for x in range(W):
            valid = [d for d in range(D) if oracle.candidate_valid(W, H, r, x, y, d)]
            if valid:
                assert abs(ds[y, x] - np.mean(valid)) < 1e-6
            else:
                assert not hv[y, x] and np.isnan(ds[y, x])


def test_lse_is_log_partition():
    H, W, D, r, tau = 12, 20, 5, 2, 0.1
    L, R = _pair(H, W, 29)
    ds, lse, hv = oracle.softargmin_fwd(L, R, 0, D, r, tau)
    y, x = 6, 12
    rho = []
    for d in range(D):
        if oracle.candidate_valid(W, H, r, x, y, d):
            a = L[y - r:y + r + 1, x - r:x + r + 1].ravel()
            b = R[y - r:y + r + 1, x - d - r:x - d + r + 1].ravel()
            rho.append((d, np.corrcoef(a, b)[0, 1]))
    z = np.array([v / tau for _, v in rho])
    assert abs(lse[y, x] - np.log(np.sum(np.exp(z)))) < 1e-12
    p = np.exp(z - lse[y, x])
    assert abs(ds[y, x] - sum(d * pi for (d, _), pi in zip(rho, p))) < 1e-12


def test_l1_loss_by_hand():
    ds = np.array([1.0, 2.0, 5.0, np.nan])
    hv = np.array([1, 1, 1, 0], np.uint8)
    gt = np.array([2.0, 2.0, 1.0, 7.0])
    loss, g = oracle.l1_loss(ds, hv, gt)
    assert loss == pytest.approx((1 + 0 + 4) / 3)
    assert g.tolist() == [-1 / 3, 0.0, 1 / 3, 0.0]
