"""Comparison helpers shared by the GPU parity tests (no method arithmetic).

Tolerances (written out in each test as well):
  * integer disparities and masks: bit-exact, except where the oracle's best
    and second-best ZNCC differ by less than NEAR_TIE (a tie that FP32
    arithmetic may break either way);
  * sub-pixel disparities: |gpu - oracle| <= 0.01 px;
  * refined disparities: relative difference <= 1e-4.
"""
import numpy as np

NEAR_TIE = 1e-5
SUB_TOL = 0.01
REFINE_RTOL = 1e-4


def to_np(t):
    return t.detach().cpu().numpy()


def int_map_mismatch(gpu, ref, exempt=None):
    """Indices where two int maps differ, outside the exempt mask."""
    diff = gpu != ref
    if exempt is not None:
        diff &= ~exempt
    return np.argwhere(diff)


def describe(idx, *maps, n=5):
    out = []
    for (y, x) in idx[:n]:
        out.append(f"({y},{x}): " + ", ".join(str(m[y, x]) for m in maps))
    return "; ".join(out)


# ------------------------------------------------------------------ full-size oracle runs
# The oracle is single-threaded; full-size workloads split it into row strips
# (each strip carries `margin` extra rows on both sides, so the rows it
# returns are exactly the full image's) evaluated by a spawn-started process
# pool (spawn: the parent may already hold a CUDA context).

def _match_strip(args):
    import oracle
    L, R, d_min, D, r, sampling, keep0, keep1 = args
    m = oracle.match(L, R, d_min, D, r, sampling)
    return {k: v[keep0:keep1] for k, v in m.items()}


def _soft_strip(args):
    import oracle
    L, R, g, d_min, D, r, tau, keep0, keep1 = args
    ds, lse, hv = oracle.softargmin_fwd(L, R, d_min, D, r, tau)
    out = dict(ds=ds[keep0:keep1], lse=lse[keep0:keep1], hv=hv[keep0:keep1])
    if g is not None:
        gL, gR = oracle.softargmin_bwd(L, R, d_min, D, r, tau, g)
        out.update(gL=gL[keep0:keep1], gR=gR[keep0:keep1])
    return out


def _procs():
    import os
    return max(1, min(32, os.cpu_count() or 1))


def _strips(H, y0, y1, n):
    rows = y1 - y0
    n = max(1, min(n, rows))
    edges = [y0 + (rows * k) // n for k in range(n + 1)]
    return [(edges[k], edges[k + 1]) for k in range(n) if edges[k + 1] > edges[k]]


def _run_pool(fn, jobs):
    import multiprocessing as mp
    if len(jobs) == 1:
        return [fn(jobs[0])]
    with mp.get_context("spawn").Pool(min(len(jobs), _procs())) as pool:
        return pool.map(fn, jobs)


def oracle_match_rows(L, R, d_min, D, r, sampling=0, y0=0, y1=None):
    """oracle.match restricted to rows [y0, y1) of the full images, evaluated
    in parallel row strips; identical to slicing oracle.match(L, R, ...)."""
    H = L.shape[0]
    y1 = H if y1 is None else y1
    jobs = []
    for a, b in _strips(H, y0, y1, 2 * _procs()):
        s0, s1 = max(0, a - r), min(H, b + r)
        jobs.append((np.ascontiguousarray(L[s0:s1]), np.ascontiguousarray(R[s0:s1]), d_min, D, r, sampling,
                     a - s0, b - s0))
    parts = _run_pool(_match_strip, jobs)
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def oracle_soft_rows(L, R, d_min, D, r, tau, g=None, y0=0, y1=None):
    """Soft-argmin forward (and, given the upstream gradient map g of the
    whole image, the image gradients) on rows [y0, y1) of full-size float
    images.  A gradient row depends on the windows of pixels up to r rows
    away, whose own windows reach r rows further: strips carry 2r margin
    rows when g is given."""
    H = L.shape[0]
    y1 = H if y1 is None else y1
    m = 2 * r if g is not None else r
    jobs = []
    for a, b in _strips(H, y0, y1, 2 * _procs()):
        s0, s1 = max(0, a - m), min(H, b + m)
        jobs.append((np.ascontiguousarray(L[s0:s1], np.float64), np.ascontiguousarray(R[s0:s1], np.float64),
                     None if g is None else np.ascontiguousarray(g[s0:s1], np.float64),
                     d_min, D, r, tau, a - s0, b - s0))
    parts = _run_pool(_soft_strip, jobs)
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


# ------------------------------------------------------------------ error report
def report(config: str, **stats):
    """Appends one JSON line of parity statistics to the file named by the
    STEREO_PARITY_REPORT environment variable (nothing when it is unset) and
    prints it (visible under pytest -s)."""
    import json
    import os
    rec = {"config": config}
    for k, v in stats.items():
        rec[k] = v.item() if hasattr(v, "item") else v
    line = json.dumps(rec, sort_keys=False)
    print("\n[parity] " + line)
    path = os.environ.get("STEREO_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")
