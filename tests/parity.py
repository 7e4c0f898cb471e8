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
