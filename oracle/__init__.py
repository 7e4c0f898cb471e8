"""FP64 CPU oracle for the dense stereo-matching path of arXiv 2007.12623, Sec. II.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by the
CPU-baseline leg of ``bench.py``; never by the product package.  The arithmetic
lives in ``oracle.c`` (plain single-threaded C, double precision, straight from
the definitions); this module only compiles it with gcc and marshals numpy
arrays through ctypes.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
library routines, invariants, brute force and hand-derived fixtures.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

INVALID = -32768
SAMPLE_FULL = 0
SAMPLE_CHESSBOARD = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (IEEE double, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
             "-ffp-contract=off", "-o", tmp, _SRC, "-lm"],
            cwd=_HERE,
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Params(C.Structure):
    _fields_ = [
        ("d_min", C.c_int), ("num_disp", C.c_int), ("win_radius", C.c_int),
        ("sampling", C.c_int), ("lr_thresh", C.c_int),
        ("outlier_rounds", C.c_int), ("r0", C.c_int), ("dr", C.c_int),
        ("outlier_thresh", C.c_double),
        ("fill_radial_r", C.c_int), ("fill_radial_min_dirs", C.c_int),
        ("fill_disc_r", C.c_int), ("fill_disc_min_count", C.c_int),
        ("smooth_radius", C.c_int), ("smooth_iters", C.c_int),
        ("alpha", C.c_double), ("eta", C.c_double), ("refine_search", C.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        i, d = C.c_int, C.c_double
        sig = {
            "or_vote_nbins": (i, [C.c_float, C.c_float]),
            "or_vote_matches": (None, [P, P, i, C.c_float, C.c_float, P, P, P]),
            "or_mosaic_frame": (i, [P, P, P, P, P, i, P, P, i, i, C.c_float, C.c_float, C.c_float, P, P,
                                    C.c_float, C.c_float, C.c_float, d, d, P, P, P]),
            "or_depth_points": (None, [P, i, i, d, d, d, d, d, P, P]),
            "or_gray": (None, [P, i, i, P]),
            "or_candidate_valid": (i, [i, i, i, i, i, i]),
            "or_zncc": (d, [P, P, i, i, i, i, i, i, i]),
            "or_cost_volume": (None, [P, P, i, i, i, i, i, i, P]),
            "or_parabola": (d, [d, d, d]),
            "or_wta_left_pixel": (i, [P, P, i, i, i, i, i, i, i, i, P, P]),
            "or_wta_right_pixel": (i, [P, P, i, i, i, i, i, i, i, i, P]),
            "or_match": (None, [P, P, i, i, i, i, i, i, P, P, P, P, P]),
            "or_lr_check": (None, [P, P, i, i, i, P]),
            "or_outlier_removal": (None, [P, i, i, i, d, P]),
            "or_fill_radial": (None, [P, i, i, i, i, P]),
            "or_disc_area": (i, [i]),
            "or_fill_disc": (None, [P, i, i, i, i, P]),
            "or_postprocess": (None, [P, i, i, i, i, i, d, i, i, i, i, P]),
            "or_refine": (None, [P, P, P, P, i, i, i, i, i, i, i, i, d, d, i, P, P]),
            "or_pipeline": (None, [P, P, i, i, P, P, P, P, P, P, P, P]),
            "or_softargmin_fwd": (None, [P, P, i, i, i, i, i, i, d, P, P, P]),
            "or_softargmin_bwd": (None, [P, P, i, i, i, i, i, i, d, P, P, P]),
            "or_l1_loss": (d, [P, P, P, C.c_size_t, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a


@dataclass
class Params:
    """Method parameters; defaults are the values of Sec. II of the paper."""
    d_min: int = 0
    num_disp: int = 32
    win_radius: int = 5              # 11x11 window (Sec. II-A)
    sampling: int = SAMPLE_FULL      # chessboard variant: Sec. II-A
    lr_thresh: int = 1               # left-right check, 1 px
    outlier_rounds: int = 3          # Sec. II-B: 3 iterations
    r0: int = 10                     # Sec. II-B: initial radius 10
    dr: int = 10                     # Sec. II-B: step 10
    outlier_thresh: float = 2.5      # Sec. II-B: smoothness threshold 2.5
    fill_radial_r: int = 50          # Sec. II-B: first hole-filling radius
    fill_radial_min_dirs: int = 4
    fill_disc_r: int = 20            # Sec. II-B: second hole-filling radius
    fill_disc_min_count: int = -1    # -1: a quarter of the disc, rounded up
    smooth_radius: int = 15          # Sec. II-C: smoothing radius 15
    smooth_iters: int = 5
    alpha: float = 0.1               # Sec. II-C, Eq. (2)
    eta: float = 0.01                # Sec. II-C, Eq. (4)
    refine_search: int = 5           # Sec. II-C: search [d-5, d+5]

    def resolved(self) -> "Params":
        q = Params(**asdict(self))
        if q.fill_disc_min_count < 0:
            q.fill_disc_min_count = (disc_area(q.fill_disc_r) + 3) // 4
        return q

    def c(self) -> _Params:
        q = self.resolved()
        return _Params(**asdict(q))


# ------------------------------------------------------------------ wrappers

def gray(rgb: np.ndarray) -> np.ndarray:
    rgb = _u8(rgb)
    H, W, _ = rgb.shape
    out = np.empty((H, W), np.uint8)
    lib().or_gray(_p(rgb), W, H, _p(out))
    return out


def candidate_valid(W, H, r, x, y, d) -> bool:
    return bool(lib().or_candidate_valid(W, H, r, x, y, d))


def zncc(L, R, r, x, y, d, sampling=SAMPLE_FULL) -> float:
    L, R = _u8(L), _u8(R)
    H, W = L.shape
    return lib().or_zncc(_p(L), _p(R), W, H, r, sampling, x, y, d)


def cost_volume(L, R, d_min, D, r, sampling=SAMPLE_FULL) -> np.ndarray:
    L, R = _u8(L), _u8(R)
    H, W = L.shape
    out = np.empty((H, W, D), np.float64)
    lib().or_cost_volume(_p(L), _p(R), W, H, d_min, D, r, sampling, _p(out))
    return out


def parabola(cm, c0, cp) -> float:
    return lib().or_parabola(cm, c0, cp)


def wta_left_pixel(L, R, d_min, D, r, x, y, sampling=SAMPLE_FULL):
    L, R = _u8(L), _u8(R)
    H, W = L.shape
    gap = C.c_double()
    sub = C.c_double()
    d = lib().or_wta_left_pixel(_p(L), _p(R), W, H, d_min, D, r, sampling, x, y,
                                C.byref(gap), C.byref(sub))
    return d, gap.value, sub.value


def wta_right_pixel(L, R, d_min, D, r, u, y, sampling=SAMPLE_FULL):
    L, R = _u8(L), _u8(R)
    H, W = L.shape
    gap = C.c_double()
    d = lib().or_wta_right_pixel(_p(L), _p(R), W, H, d_min, D, r, sampling, u, y,
                                 C.byref(gap))
    return d, gap.value


def match(L, R, d_min, D, r, sampling=SAMPLE_FULL):
    """Winner-take-all maps: dict(dL, dR, sub, gapL, gapR)."""
    L, R = _u8(L), _u8(R)
    H, W = L.shape
    out = dict(dL=np.empty((H, W), np.int16), dR=np.empty((H, W), np.int16),
               sub=np.empty((H, W)), gapL=np.empty((H, W)), gapR=np.empty((H, W)))
    lib().or_match(_p(L), _p(R), W, H, d_min, D, r, sampling, _p(out["dL"]),
                   _p(out["dR"]), _p(out["sub"]), _p(out["gapL"]), _p(out["gapR"]))
    return out


def lr_check(dL, dR, thresh=1):
    dL = np.ascontiguousarray(dL, np.int16)
    dR = np.ascontiguousarray(dR, np.int16)
    H, W = dL.shape
    out = np.empty_like(dL)
    lib().or_lr_check(_p(dL), _p(dR), W, H, thresh, _p(out))
    return out


def outlier_removal(o, radius, thresh=2.5):
    o = np.ascontiguousarray(o, np.int16)
    H, W = o.shape
    out = np.empty_like(o)
    lib().or_outlier_removal(_p(o), W, H, radius, thresh, _p(out))
    return out


def fill_radial(o, radius=50, min_dirs=4):
    o = np.ascontiguousarray(o, np.int16)
    H, W = o.shape
    out = np.empty_like(o)
    lib().or_fill_radial(_p(o), W, H, radius, min_dirs, _p(out))
    return out


def disc_area(radius) -> int:
    return lib().or_disc_area(radius)


def fill_disc(o, radius=20, min_count=None):
    o = np.ascontiguousarray(o, np.int16)
    H, W = o.shape
    if min_count is None:
        min_count = (disc_area(radius) + 3) // 4
    out = np.empty_like(o)
    lib().or_fill_disc(_p(o), W, H, radius, min_count, _p(out))
    return out


def postprocess(o, p: Params = Params()):
    q = p.resolved()
    o = np.ascontiguousarray(o, np.int16)
    H, W = o.shape
    out = np.empty_like(o)
    lib().or_postprocess(_p(o), W, H, q.outlier_rounds, q.r0, q.dr, q.outlier_thresh,
                         q.fill_radial_r, q.fill_radial_min_dirs, q.fill_disc_r,
                         q.fill_disc_min_count, _p(out))
    return out


def refine(o, cost=None, L=None, R=None, p: Params = Params()):
    """Improved Laplacian refinement, Sec. II-C.  Returns (d^(K), o_final).

    ``cost`` is a [H, W, D] volume of 1 - ZNCC (NaN = invalid candidate); when
    it is None the ZNCC is computed from ``L``/``R`` by the definition.
    """
    q = p.resolved()
    o = np.ascontiguousarray(o, np.int16)
    H, W = o.shape
    if cost is not None:
        cost = np.ascontiguousarray(cost, np.float64)
        assert cost.shape == (H, W, q.num_disp)
    if L is not None:
        L, R = _u8(L), _u8(R)
    d_out = np.empty((H, W))
    o_out = np.empty_like(o)
    lib().or_refine(_p(o), _p(cost), _p(L), _p(R), W, H, q.d_min, q.num_disp,
                    q.win_radius, q.sampling, q.smooth_radius, q.smooth_iters,
                    q.alpha, q.eta, q.refine_search, _p(d_out), _p(o_out))
    return d_out, o_out


def pipeline(L, R, p: Params):
    """Whole path S2-S7.  Returns a dict of every stage's output."""
    L, R = _u8(L), _u8(R)
    H, W = L.shape
    D = p.num_disp
    out = dict(dL=np.empty((H, W), np.int16), dR=np.empty((H, W), np.int16),
               sub=np.empty((H, W)), o_lr=np.empty((H, W), np.int16),
               o_post=np.empty((H, W), np.int16), d_final=np.empty((H, W)),
               cost=np.empty((H, W, D)))
    pc = p.c()
    lib().or_pipeline(_p(L), _p(R), W, H, C.byref(pc), _p(out["dL"]), _p(out["dR"]),
                      _p(out["sub"]), _p(out["o_lr"]), _p(out["o_post"]),
                      _p(out["d_final"]), _p(out["cost"]))
    return out


def softargmin_fwd(L, R, d_min, D, r, tau, sampling=SAMPLE_FULL):
    L = np.ascontiguousarray(L, np.float64)
    R = np.ascontiguousarray(R, np.float64)
    H, W = L.shape
    ds = np.empty((H, W))
    lse = np.empty((H, W))
    hv = np.empty((H, W), np.uint8)
    lib().or_softargmin_fwd(_p(L), _p(R), W, H, d_min, D, r, sampling, tau,
                            _p(ds), _p(lse), _p(hv))
    return ds, lse, hv.astype(bool)


def softargmin_bwd(L, R, d_min, D, r, tau, grad_dsoft, sampling=SAMPLE_FULL):
    L = np.ascontiguousarray(L, np.float64)
    R = np.ascontiguousarray(R, np.float64)
    g = np.ascontiguousarray(grad_dsoft, np.float64)
    H, W = L.shape
    gL = np.empty((H, W))
    gR = np.empty((H, W))
    lib().or_softargmin_bwd(_p(L), _p(R), W, H, d_min, D, r, sampling, tau, _p(g),
                            _p(gL), _p(gR))
    return gL, gR


def l1_loss(dsoft, has_valid, gt):
    ds = np.ascontiguousarray(dsoft, np.float64).ravel()
    hv = np.ascontiguousarray(has_valid, np.uint8).ravel()
    gt = np.ascontiguousarray(gt, np.float64).ravel()
    g = np.empty_like(ds)
    loss = lib().or_l1_loss(_p(ds), _p(hv), _p(gt), ds.size, _p(g))
    return loss, g.reshape(np.shape(dsoft))


def depth_points(disp, f, cx, cy, B, doffs=0.0):
    """Disparity -> points and normals in the left camera frame (Sec. II,
    reprojection of a rectified pair).  Returns (xyz [H, W, 3], normals
    [H, W, 3]), NaN where undefined."""
    d = np.ascontiguousarray(disp, np.float64)
    H, W = d.shape
    xyz = np.empty((H, W, 3))
    nrm = np.empty((H, W, 3))
    lib().or_depth_points(_p(d), W, H, float(f), float(cx), float(cy), float(B), float(doffs),
                          _p(xyz), _p(nrm))
    return xyz, nrm


class PointModel:
    """The mosaicked surface model of the oracle: float64 arrays of a fixed
    capacity and the number of points in use."""

    def __init__(self, capacity: int):
        self.pos = np.zeros((capacity, 3))
        self.rgb = np.zeros((capacity, 3))
        self.wpos = np.zeros(capacity)
        self.wrgb = np.zeros(capacity)
        self.count = 0
        self.capacity = capacity


def mosaic_frame(model: PointModel, xyz, img, f, cx, cy, R, t, tau, r0=0.5, gmin=0.1, margins=None):
    """Point-based TSDF mosaicking of one frame (Sec. II), in double
    precision; updates `model` in place and returns the number of appends
    that did not fit.

    margins=(eps_pix, eps_rel) also returns the decision margins as a second
    value: dict(fragile_pix [H, W] bool, fragile_pt [n] bool for the points
    the model held before the frame, src_pixel [count] int: the pixel each
    appended point came from, -1 for older points)."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    img = np.ascontiguousarray(img, np.uint8)
    H, W = xyz.shape[:2]
    R = np.ascontiguousarray(R, np.float32).reshape(9)
    t = np.ascontiguousarray(t, np.float32).reshape(3)
    n0 = model.count
    cnt = C.c_int(model.count)
    fp = fq = src = None
    eps_pix, eps_rel = margins if margins is not None else (0.0, 0.0)
    if margins is not None:
        fp = np.zeros((H, W), np.uint8)
        fq = np.zeros(max(n0, 1), np.uint8)
        src = np.full(model.capacity, -1, np.int32)
    dropped = lib().or_mosaic_frame(_p(model.pos), _p(model.rgb), _p(model.wpos), _p(model.wrgb),
                                    C.byref(cnt), model.capacity, _p(xyz), _p(img), W, H, float(f),
                                    float(cx), float(cy), _p(R), _p(t), float(tau), float(r0), float(gmin),
                                    float(eps_pix), float(eps_rel), _p(fp), _p(fq), _p(src))
    model.count = cnt.value
    if margins is None:
        return dropped
    return dropped, dict(fragile_pix=fp.astype(bool), fragile_pt=fq[:n0].astype(bool),
                         src_pixel=src[:model.count])


def vote_matches(uv1, uv2, bin=4.0, range_=128.0):
    """Histogram-voting preselection (Sec. II): returns (hist [nb, nb],
    score [n], order [n])."""
    uv1 = np.ascontiguousarray(uv1, np.float32)
    uv2 = np.ascontiguousarray(uv2, np.float32)
    n = uv1.shape[0]
    nb = lib().or_vote_nbins(float(bin), float(range_))
    hist = np.empty((nb, nb), np.int32)
    score = np.empty(n, np.int32)
    order = np.empty(n, np.int32)
    lib().or_vote_matches(_p(uv1), _p(uv2), n, float(bin), float(range_), _p(hist), _p(score), _p(order))
    return hist, score, order
