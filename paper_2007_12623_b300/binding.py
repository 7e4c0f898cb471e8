"""ctypes binding of include/stereo.h.  Same names as the C ABI; arguments are
torch tensors (device memory) and an optional torch/CUDA stream.  Nothing here
computes: it checks dtypes/devices, takes data pointers and calls the
library."""
from __future__ import annotations

import ctypes as C
import os
import re

from . import build as _build

__all__ = [
    "INVALID", "COST_NONE", "COST_F32", "COST_F16", "COST_BF16", "SAMPLE_FULL",
    "SAMPLE_CHESSBOARD", "STATUS", "StereoError", "StereoParams", "StereoPair", "Handle", "lib",
    "lib_path", "header_functions", "cost_stride", "stereo_default_params", "stereo_create",
    "stereo_destroy", "stereo_match", "stereo_match_batched", "stereo_get_device_error",
    "stereo_status_str", "stereo_gray", "stereo_stage_match", "stereo_stage_lr",
    "stereo_stage_outlier", "stereo_stage_fill_radial", "stereo_stage_fill_disc",
    "stereo_stage_postprocess", "stereo_stage_refine", "stereo_set_stage_timing",
    "stereo_get_stage_times", "stereo_launch_count", "STAGE_NAMES", "stereo_set_tuning",
    "stereo_match_wta_noalloc", "stereo_softargmin_fwd", "stereo_softargmin_bwd", "stereo_l1_loss",
    "SoftArgminZNCC", "soft_argmin", "stereo_set_batch_config", "stereo_autotune_batched",
    "stereo_set_batch_stages", "stereo_get_batch_config", "checked_library", "stereo_debug_fail_alloc",
    "stereo_debug_live_allocations",
    "StereoCamera", "stereo_depth_points", "PointModel", "stereo_mosaic_frame", "stereo_vote_nbins",
    "stereo_vote_matches",
]

STAGE_NAMES = ("input", "stats", "cost_wta", "finalize", "postprocess", "refine")

INVALID = -32768
COST_NONE, COST_F32, COST_F16, COST_BF16 = 0, 1, 2, 3
SAMPLE_FULL, SAMPLE_CHESSBOARD = 0, 1
STATUS = {0: "STEREO_OK", 1: "STEREO_ERR_INVALID_ARG", 2: "STEREO_ERR_CUDA", 3: "STEREO_ERR_OOM",
          4: "STEREO_ERR_UNSUPPORTED", 5: "STEREO_ERR_TIMEOUT", 6: "STEREO_ERR_TOO_LARGE"}

_HEADER = os.path.join(os.path.dirname(_build.HERE), "include", "stereo.h")


class StereoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class StereoParams(C.Structure):
    _fields_ = [
        ("max_width", C.c_int32), ("max_height", C.c_int32),
        ("d_min", C.c_int32), ("num_disp", C.c_int32),
        ("win_radius", C.c_int32), ("sampling", C.c_int32), ("cost_dtype", C.c_int32),
        ("lr_thresh", C.c_int32),
        ("outlier_rounds", C.c_int32), ("r0", C.c_int32), ("dr", C.c_int32),
        ("outlier_thresh", C.c_float),
        ("fill_radial_r", C.c_int32), ("fill_radial_min_dirs", C.c_int32),
        ("fill_disc_r", C.c_int32), ("fill_disc_min_count", C.c_int32),
        ("smooth_radius", C.c_int32), ("smooth_iters", C.c_int32),
        ("alpha", C.c_float), ("eta", C.c_float), ("refine_search", C.c_int32),
        ("soft_argmin", C.c_int32),
    ]


class StereoPair(C.Structure):
    _fields_ = [
        ("left", C.c_void_p), ("right", C.c_void_p),
        ("width", C.c_int32), ("height", C.c_int32), ("pitch", C.c_int32), ("channels", C.c_int32),
        ("disp_wta", C.c_void_p), ("disp_sub", C.c_void_p), ("disp_lr", C.c_void_p),
        ("disp_post", C.c_void_p), ("valid", C.c_void_p), ("disp_final", C.c_void_p),
        ("d_min", C.c_int32), ("num_disp", C.c_int32), ("win_radius", C.c_int32),
    ]


class StereoCamera(C.Structure):
    _fields_ = [("f", C.c_float), ("cx", C.c_float), ("cy", C.c_float), ("baseline", C.c_float),
                ("doffs", C.c_float)]


class _PointModelC(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("rgb", C.c_void_p), ("wpos", C.c_void_p), ("wrgb", C.c_void_p),
                ("count", C.c_void_p), ("dropped", C.c_void_p), ("capacity", C.c_int32)]





_libs = {}
_use_checked = False


def lib_path() -> str:
    return _build.LIB_CHECKED if _use_checked else _build.LIB


class checked_library:
    """Context in which every call of this binding goes to the checked build
    (libstereo_checked.so: in-kernel index checks that record a failure in
    the device error word and skip the access).  Handles belong to the
    library that created them: create, use and close them inside the same
    context."""

    def __enter__(self):
        global _use_checked
        self._prev = _use_checked
        _use_checked = True
        return lib()

    def __exit__(self, *exc):
        global _use_checked
        _use_checked = self._prev


def lib():
    """Loads libstereo.so (or, inside checked_library, libstereo_checked.so);
    raises if it has not been built."""
    path = lib_path()
    if path not in _libs:
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not built ({path}); run "
                               "python -m paper_2007_12623_b300.build")
        L = C.CDLL(path)
        P, i32, f32 = C.c_void_p, C.c_int32, C.c_float
        sig = {
            "stereo_default_params": (None, [P]),
            "stereo_create": (C.c_int, [P, i32, P]),
            "stereo_destroy": (C.c_int, [P]),
            "stereo_match": (C.c_int, [P, P, P]),
            "stereo_match_batched": (C.c_int, [P, P, i32, i32, P]),
            "stereo_get_device_error": (C.c_int, [P, P, P]),
            "stereo_status_str": (C.c_char_p, [C.c_int]),
            "stereo_gray": (C.c_int, [P, i32, i32, i32, P, P]),
            "stereo_stage_match": (C.c_int, [P, P, P, i32, i32, i32, i32, i32, i32, i32, P, P, P, P, P]),
            "stereo_stage_lr": (C.c_int, [P, P, i32, i32, i32, P, P]),
            "stereo_stage_outlier": (C.c_int, [P, P, i32, i32, i32, f32, P, P]),
            "stereo_stage_fill_radial": (C.c_int, [P, P, i32, i32, i32, i32, P, P]),
            "stereo_stage_fill_disc": (C.c_int, [P, P, i32, i32, i32, i32, P, P]),
            "stereo_stage_postprocess": (C.c_int, [P, P, i32, i32, P, P]),
            "stereo_stage_refine": (C.c_int, [P, P, P, i32, P, P, i32, i32, i32, i32, i32, P, P, P]),
            "stereo_set_stage_timing": (C.c_int, [P, i32]),
            "stereo_get_stage_times": (C.c_int, [P, P, i32]),
            "stereo_launch_count": (C.c_ulonglong, []),
            "stereo_set_tuning": (C.c_int, [C.c_char_p, i32]),
            "stereo_match_wta_noalloc": (C.c_int, [P, P, i32, i32, i32, i32, i32, P, P, P, P]),
            "stereo_softargmin_fwd": (C.c_int, [P, P, P, i32, i32, i32, i32, i32, i32, f32, P, P, P]),
            "stereo_softargmin_bwd": (C.c_int, [P, P, P, i32, i32, i32, i32, i32, i32, f32, P, P, P, P, P,
                                                P]),
            "stereo_l1_loss": (C.c_int, [P, P, P, C.c_int64, P, P, P]),
            "stereo_depth_points": (C.c_int, [P, i32, i32, P, P, P, P]),
            "stereo_vote_nbins": (i32, [C.c_float, C.c_float]),
            "stereo_vote_matches": (C.c_int, [P, P, i32, C.c_float, C.c_float, P, P, P, P]),
            "stereo_mosaic_frame": (C.c_int, [P, P, P, P, i32, i32, P, P, P, C.c_float, C.c_float,
                                              C.c_float, P]),
            "stereo_set_batch_config": (C.c_int, [P, i32, i32]),
            "stereo_set_batch_stages": (C.c_int, [P, i32]),
            "stereo_get_batch_config": (C.c_int, [P, P, P, P]),
            "stereo_autotune_batched": (C.c_int, [P, P, i32, P, P, P, P]),
            "stereo_debug_fail_alloc": (C.c_int, [i32]),
            "stereo_debug_live_allocations": (C.c_int64, []),
            "stereo_build_checked": (i32, []),
            "stereo_debug_check_selftest": (C.c_int, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _libs[path] = L
    return _libs[path]


def header_functions() -> list[str]:
    """Names of the functions declared in include/stereo.h."""
    txt = open(_HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(stereo_[a-z_]+)\s*\(", txt)))


def cost_stride(num_disp: int) -> int:
    """Elements per pixel in a cost volume (num_disp rounded up to 8)."""
    return (num_disp + 7) & ~7


# ------------------------------------------------------------- marshalling

def _check(status: int, where: str):
    if status != 0:
        raise StereoError(status, where)


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _cost_torch_dtype(cdt):
    import torch
    return {COST_F32: torch.float32, COST_F16: torch.float16, COST_BF16: torch.bfloat16}.get(cdt)


# ------------------------------------------------------------------ API

def stereo_default_params(**overrides) -> StereoParams:
    p = StereoParams()
    lib().stereo_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Handle:
    """Owns a stereo_handle; destroyed by close() or garbage collection."""

    def __init__(self, ptr, params: StereoParams, max_batch: int):
        self.ptr = ptr
        self.params = params
        self.max_batch = max_batch
        self._lib = lib()               # the library that created it destroys it

    def close(self):
        if self.ptr:
            self._lib.stereo_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stereo_create(params: StereoParams, max_batch: int = 1) -> Handle:
    h = C.c_void_p()
    _check(lib().stereo_create(C.byref(params), max_batch, C.byref(h)), "stereo_create")
    return Handle(h, params, max_batch)


def stereo_destroy(handle: Handle):
    handle.close()


def _pair_struct(left, right, disp_wta=None, disp_sub=None, disp_lr=None, disp_post=None,
                 valid=None, disp_final=None, d_min=0, num_disp=0, win_radius=0):
    import torch
    if left.dim() == 3:
        H, W, ch = left.shape
    else:
        (H, W), ch = left.shape, 1
    if right.shape != left.shape:
        raise ValueError("left/right shapes differ")
    p = StereoPair()
    p.left = _ptr(left, torch.uint8, "left")
    p.right = _ptr(right, torch.uint8, "right")
    p.width, p.height, p.pitch, p.channels = W, H, W * ch, ch
    p.disp_wta = _ptr(disp_wta, torch.int16, "disp_wta")
    p.disp_sub = _ptr(disp_sub, torch.float32, "disp_sub")
    p.disp_lr = _ptr(disp_lr, torch.int16, "disp_lr")
    p.disp_post = _ptr(disp_post, torch.int16, "disp_post")
    p.valid = _ptr(valid, torch.uint8, "valid")
    p.disp_final = _ptr(disp_final, torch.float32, "disp_final")
    p.d_min, p.num_disp, p.win_radius = d_min, num_disp, win_radius
    return p


def stereo_match(handle: Handle, left, right, *, disp_wta=None, disp_sub=None, disp_lr=None,
                 disp_post=None, valid=None, disp_final=None, d_min=0, num_disp=0, win_radius=0,
                 stream=None):
    """Whole path on one pair (uint8 HxW gray or HxWx3 RGB tensors)."""
    p = _pair_struct(left, right, disp_wta, disp_sub, disp_lr, disp_post, valid, disp_final,
                     d_min, num_disp, win_radius)
    _check(lib().stereo_match(handle.ptr, C.byref(p), _stream(stream)), "stereo_match")


def _pair_array(pairs):
    arr = (StereoPair * len(pairs))()
    for i, d in enumerate(pairs):
        arr[i] = _pair_struct(**d)
    return arr


def stereo_match_batched(handle: Handle, pairs, use_graph: bool = True, stream=None):
    """pairs: list of dicts with the keyword arguments of stereo_match plus
    left/right (per-pair d_min / num_disp / win_radius allowed)."""
    arr = _pair_array(pairs)
    _check(lib().stereo_match_batched(handle.ptr, arr, len(pairs), int(bool(use_graph)),
                                      _stream(stream)), "stereo_match_batched")


def stereo_set_batch_config(handle: Handle, rows: int = 0, K: int = 0):
    _check(lib().stereo_set_batch_config(handle.ptr, rows, K), "stereo_set_batch_config")


def stereo_set_batch_stages(handle: Handle, mode: int = 0):
    _check(lib().stereo_set_batch_stages(handle.ptr, mode), "stereo_set_batch_stages")


def stereo_get_batch_config(handle: Handle) -> dict:
    rows, K, stages = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().stereo_get_batch_config(handle.ptr, C.byref(rows), C.byref(K), C.byref(stages)),
           "stereo_get_batch_config")
    return dict(rows=rows.value, K=K.value, stages=stages.value)


def stereo_autotune_batched(handle: Handle, pairs, stream=None):
    """Times the batched cost stage for each candidate unit configuration and
    both stage modes, and keeps the fastest; returns dict(rows, K, ms,
    stages)."""
    arr = _pair_array(pairs)
    rows, K, ms = C.c_int32(), C.c_int32(), C.c_float()
    _check(lib().stereo_autotune_batched(handle.ptr, arr, len(pairs), _stream(stream), C.byref(rows),
                                         C.byref(K), C.byref(ms)), "stereo_autotune_batched")
    return dict(rows=rows.value, K=K.value, ms=ms.value, stages=stereo_get_batch_config(handle)["stages"])


def stereo_get_device_error(handle: Handle, stream=None) -> int:
    e = C.c_int32()
    _check(lib().stereo_get_device_error(handle.ptr, C.byref(e), _stream(stream)),
           "stereo_get_device_error")
    return e.value


def stereo_debug_fail_alloc(n: int):
    """Test hook: the device allocation n + 1 calls later fails as if the
    device were out of memory (-1 disarms)."""
    _check(lib().stereo_debug_fail_alloc(n), "stereo_debug_fail_alloc")


def stereo_debug_live_allocations() -> int:
    return int(lib().stereo_debug_live_allocations())


def stereo_status_str(status: int) -> str:
    return lib().stereo_status_str(status).decode()


def stereo_gray(rgb, gray, stream=None):
    import torch
    H, W, _ = rgb.shape
    _check(lib().stereo_gray(_ptr(rgb, torch.uint8, "rgb"), W, H, 3 * W,
                             _ptr(gray, torch.uint8, "gray"), _stream(stream)), "stereo_gray")


def stereo_stage_match(handle: Handle, left, right, d_min, num_disp, win_radius, sampling,
                       cost_dtype, disp_left, disp_right, disp_sub, cost=None, stream=None):
    import torch
    H, W = left.shape
    _check(lib().stereo_stage_match(
        handle.ptr, _ptr(left, torch.uint8, "left"), _ptr(right, torch.uint8, "right"), W, H,
        d_min, num_disp, win_radius, sampling, cost_dtype,
        _ptr(disp_left, torch.int16, "disp_left"), _ptr(disp_right, torch.int16, "disp_right"),
        _ptr(disp_sub, torch.float32, "disp_sub"), _ptr(cost, _cost_torch_dtype(cost_dtype), "cost"),
        _stream(stream)), "stereo_stage_match")


def stereo_stage_lr(disp_left, disp_right, thresh, out, stream=None):
    import torch
    H, W = disp_left.shape
    _check(lib().stereo_stage_lr(_ptr(disp_left, torch.int16), _ptr(disp_right, torch.int16), W, H,
                                 thresh, _ptr(out, torch.int16), _stream(stream)), "stereo_stage_lr")


def stereo_stage_outlier(handle: Handle, inp, radius, thresh, out, stream=None):
    import torch
    H, W = inp.shape
    _check(lib().stereo_stage_outlier(handle.ptr, _ptr(inp, torch.int16), W, H, radius, thresh,
                                      _ptr(out, torch.int16), _stream(stream)),
           "stereo_stage_outlier")


def stereo_stage_fill_radial(handle: Handle, inp, radius, min_dirs, out, stream=None):
    import torch
    H, W = inp.shape
    _check(lib().stereo_stage_fill_radial(handle.ptr, _ptr(inp, torch.int16), W, H, radius, min_dirs,
                                          _ptr(out, torch.int16), _stream(stream)),
           "stereo_stage_fill_radial")


def stereo_stage_fill_disc(handle: Handle, inp, radius, min_count, out, stream=None):
    import torch
    H, W = inp.shape
    _check(lib().stereo_stage_fill_disc(handle.ptr, _ptr(inp, torch.int16), W, H, radius, min_count,
                                        _ptr(out, torch.int16), _stream(stream)),
           "stereo_stage_fill_disc")


def stereo_stage_postprocess(handle: Handle, inp, out, stream=None):
    import torch
    H, W = inp.shape
    _check(lib().stereo_stage_postprocess(handle.ptr, _ptr(inp, torch.int16), W, H,
                                          _ptr(out, torch.int16), _stream(stream)),
           "stereo_stage_postprocess")


def stereo_stage_refine(handle: Handle, o_in, cost, cost_dtype, left, right, d_min, num_disp,
                        win_radius, d_out, o_out=None, stream=None):
    import torch
    H, W = o_in.shape
    _check(lib().stereo_stage_refine(
        handle.ptr, _ptr(o_in, torch.int16, "o_in"), _ptr(cost, _cost_torch_dtype(cost_dtype), "cost"),
        cost_dtype, _ptr(left, torch.uint8, "left"), _ptr(right, torch.uint8, "right"), W, H, d_min,
        num_disp, win_radius, _ptr(d_out, torch.float32, "d_out"), _ptr(o_out, torch.int16, "o_out"),
        _stream(stream)), "stereo_stage_refine")


def stereo_set_stage_timing(handle: Handle, enable: bool = True):
    _check(lib().stereo_set_stage_timing(handle.ptr, int(bool(enable))), "stereo_set_stage_timing")


def stereo_get_stage_times(handle: Handle) -> dict:
    """Per-stage milliseconds of the handle's last stereo_match (waits for it)."""
    arr = (C.c_float * len(STAGE_NAMES))()
    _check(lib().stereo_get_stage_times(handle.ptr, arr, len(STAGE_NAMES)), "stereo_get_stage_times")
    return dict(zip(STAGE_NAMES, [float(v) for v in arr]))


def stereo_launch_count() -> int:
    return int(lib().stereo_launch_count())


def stereo_set_tuning(name: str, value: int):
    """Process-wide tuning knob (see include/stereo.h), 0 = automatic."""
    _check(lib().stereo_set_tuning(name.encode(), int(value)), "stereo_set_tuning")


def stereo_match_wta_noalloc(left, right, d_min, num_disp, win_radius, disp_left, disp_right,
                             disp_sub=None, stream=None):
    """Cost + winner-take-all without any allocation (fixed in-library scratch);
    see include/stereo.h for the limits and the no-overlap rule."""
    import torch
    H, W = left.shape
    _check(lib().stereo_match_wta_noalloc(
        _ptr(left, torch.uint8, "left"), _ptr(right, torch.uint8, "right"), W, H, d_min, num_disp,
        win_radius, _ptr(disp_left, torch.int16, "disp_left"), _ptr(disp_right, torch.int16, "disp_right"),
        _ptr(disp_sub, torch.float32, "disp_sub"), _stream(stream)), "stereo_match_wta_noalloc")


# ------------------------------------------------------------ soft-argmin

def _bhw(t):
    if t.dim() == 2:
        return 1, t.shape[0], t.shape[1]
    return t.shape[0], t.shape[1], t.shape[2]


def stereo_softargmin_fwd(handle: Handle, left, right, d_min, num_disp, win_radius, tau, d_soft, lse,
                          stream=None):
    import torch
    B, H, W = _bhw(left)
    _check(lib().stereo_softargmin_fwd(
        handle.ptr, _ptr(left, torch.float32, "left"), _ptr(right, torch.float32, "right"), B, W, H,
        d_min, num_disp, win_radius, tau, _ptr(d_soft, torch.float32, "d_soft"),
        _ptr(lse, torch.float32, "lse"), _stream(stream)), "stereo_softargmin_fwd")


def stereo_softargmin_bwd(handle: Handle, left, right, d_min, num_disp, win_radius, tau, d_soft, lse,
                          grad_dsoft, grad_left, grad_right, stream=None):
    import torch
    B, H, W = _bhw(left)
    _check(lib().stereo_softargmin_bwd(
        handle.ptr, _ptr(left, torch.float32, "left"), _ptr(right, torch.float32, "right"), B, W, H,
        d_min, num_disp, win_radius, tau, _ptr(d_soft, torch.float32, "d_soft"),
        _ptr(lse, torch.float32, "lse"), _ptr(grad_dsoft, torch.float32, "grad_dsoft"),
        _ptr(grad_left, torch.float32, "grad_left"), _ptr(grad_right, torch.float32, "grad_right"),
        _stream(stream)), "stereo_softargmin_bwd")


def stereo_l1_loss(handle: Handle, d_soft, gt, loss, grad=None, stream=None):
    import torch
    _check(lib().stereo_l1_loss(handle.ptr, _ptr(d_soft, torch.float32, "d_soft"), _ptr(gt, torch.float32, "gt"),
                                d_soft.numel(), _ptr(loss, torch.float32, "loss"),
                                _ptr(grad, torch.float32, "grad"), _stream(stream)), "stereo_l1_loss")


def stereo_depth_points(disp, camera: StereoCamera, xyz=None, normals=None, stream=None):
    """Sec. II depth from disparity: points and normals [H, W, 3] (float32,
    NaN where undefined) of a float disparity map [H, W]."""
    import torch
    H, W = disp.shape
    for name, t in (("xyz", xyz), ("normals", normals)):
        if t is not None and tuple(t.shape) != (H, W, 3):
            raise ValueError(f"{name}: expected shape {(H, W, 3)}")
    _check(lib().stereo_depth_points(_ptr(disp, torch.float32, "disp"), W, H, C.byref(camera),
                                     _ptr(xyz, torch.float32, "xyz"), _ptr(normals, torch.float32, "normals"),
                                     _stream(stream)), "stereo_depth_points")


def stereo_vote_nbins(bin: float, range_: float) -> int:
    return int(lib().stereo_vote_nbins(float(bin), float(range_)))


def stereo_vote_matches(uv1, uv2, bin=4.0, range_=128.0, hist=None, score=None, order=None, stream=None):
    """Histogram-voting inlier preselection (Sec. II) of n matches (uv1, uv2:
    float32 [n, 2] device tensors).  Returns (hist [nb, nb], score [n],
    order [n]) int32 device tensors."""
    import torch
    n = uv1.shape[0]
    nb = stereo_vote_nbins(bin, range_)
    hist = hist if hist is not None else torch.empty((nb, nb), dtype=torch.int32, device=uv1.device)
    score = score if score is not None else torch.empty(n, dtype=torch.int32, device=uv1.device)
    order = order if order is not None else torch.empty(n, dtype=torch.int32, device=uv1.device)
    _check(lib().stereo_vote_matches(_ptr(uv1, torch.float32, "uv1"), _ptr(uv2, torch.float32, "uv2"), n,
                                     float(bin), float(range_), _ptr(hist, torch.int32, "hist"),
                                     _ptr(score, torch.int32, "score"), _ptr(order, torch.int32, "order"),
                                     _stream(stream)), "stereo_vote_matches")
    return hist, score, order


class PointModel:
    """Device arrays of a mosaicked surface model (torch tensors): pos, rgb
    [capacity, 3], wpos, wrgb [capacity] (float32), count, dropped (int32
    scalars on the device)."""

    def __init__(self, capacity: int, device):
        import torch
        self.capacity = capacity
        self.pos = torch.zeros((capacity, 3), dtype=torch.float32, device=device)
        self.rgb = torch.zeros((capacity, 3), dtype=torch.float32, device=device)
        self.wpos = torch.zeros(capacity, dtype=torch.float32, device=device)
        self.wrgb = torch.zeros(capacity, dtype=torch.float32, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)
        self.dropped = torch.zeros(1, dtype=torch.int32, device=device)

    def _c(self):
        return _PointModelC(self.pos.data_ptr(), self.rgb.data_ptr(), self.wpos.data_ptr(),
                            self.wrgb.data_ptr(), self.count.data_ptr(), self.dropped.data_ptr(),
                            self.capacity)


def stereo_mosaic_frame(handle: Handle, model: PointModel, xyz, rgb, camera: StereoCamera, R, t, tau,
                        r0=0.5, gmin=0.1, stream=None):
    """Point-based TSDF mosaicking of one key frame (Sec. II): xyz [H, W, 3]
    float32 camera-frame points (NaN = no depth), rgb [H, W, 3] uint8, R (3x3)
    and t (3) the world-to-camera pose."""
    import torch
    H, W = xyz.shape[:2]
    import numpy as np
    Rf = (C.c_float * 9)(*np.asarray(R, dtype=np.float32).reshape(9).tolist())
    tf = (C.c_float * 3)(*np.asarray(t, dtype=np.float32).reshape(3).tolist())
    mc = model._c()
    _check(lib().stereo_mosaic_frame(handle.ptr, C.byref(mc), _ptr(xyz, torch.float32, "xyz"),
                                     _ptr(rgb, torch.uint8, "rgb"), W, H, C.byref(camera), Rf, tf, float(tau),
                                     float(r0), float(gmin), _stream(stream)), "stereo_mosaic_frame")


def _autograd_function():
    import torch

    class SoftArgminZNCC(torch.autograd.Function):
        """d_soft = soft-argmin over disparities of ZNCC / tau (float images,
        [B,] H, W).  Forward and backward both run in libstereo; the backward
        recomputes the window statistics and ZNCC."""

        @staticmethod
        def forward(ctx, left, right, handle, d_min, num_disp, win_radius, tau):
            left = left.contiguous()
            right = right.contiguous()
            d_soft = torch.empty_like(left)
            lse = torch.empty_like(left)
            stereo_softargmin_fwd(handle, left, right, d_min, num_disp, win_radius, tau, d_soft, lse)
            ctx.save_for_backward(left, right, d_soft, lse)
            ctx.cfg = (handle, d_min, num_disp, win_radius, tau)
            return d_soft

        @staticmethod
        def backward(ctx, grad_dsoft):
            left, right, d_soft, lse = ctx.saved_tensors
            handle, d_min, num_disp, win_radius, tau = ctx.cfg
            g = torch.nan_to_num(grad_dsoft.contiguous(), nan=0.0)
            gl = torch.empty_like(left)
            gr = torch.empty_like(right)
            stereo_softargmin_bwd(handle, left, right, d_min, num_disp, win_radius, tau, d_soft, lse, g,
                                  gl, gr)
            return gl, gr, None, None, None, None, None

    return SoftArgminZNCC


class _LazyFn:
    _fn = None

    def __get__(self, obj, objtype=None):
        if _LazyFn._fn is None:
            _LazyFn._fn = _autograd_function()
        return _LazyFn._fn


class _Namespace:
    SoftArgminZNCC = _LazyFn()


def __getattr__(name):
    if name == "SoftArgminZNCC":
        return _Namespace.SoftArgminZNCC
    raise AttributeError(name)


def soft_argmin(left, right, handle: Handle, d_min=0, num_disp=128, win_radius=5, tau=0.1):
    """Differentiable soft-argmin disparity (torch autograd)."""
    return _Namespace.SoftArgminZNCC.apply(left, right, handle, d_min, num_disp, win_radius, tau)
