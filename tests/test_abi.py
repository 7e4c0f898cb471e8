"""Host-side checks of the C ABI: the library loads without a GPU, exports
every function include/stereo.h declares, carries the paper's defaults and
rejects bad arguments on the host before touching the device."""
import ctypes as C

import pytest

import paper_2007_12623_b300 as st
from paper_2007_12623_b300 import build as stbuild


@pytest.fixture(scope="module")
def L():
    stbuild.build()
    return st.lib()


def test_exports_every_declared_function(L):
    names = st.header_functions()
    assert "stereo_match" in names and "stereo_create" in names and "stereo_destroy" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_default_params_are_the_papers():
    p = st.stereo_default_params()
    assert p.win_radius == 5                      # 11x11 window, Sec. II-A
    assert p.outlier_thresh == 2.5                # Sec. II-B
    assert (p.outlier_rounds, p.r0, p.dr) == (3, 10, 10)
    assert (p.fill_radial_r, p.fill_disc_r) == (50, 20)
    assert p.smooth_radius == 15                  # Sec. II-C
    assert abs(p.alpha - 0.1) < 1e-7 and abs(p.eta - 0.01) < 1e-9
    assert p.refine_search == 5
    assert p.lr_thresh == 1


def test_status_strings(L):
    assert st.stereo_status_str(0) == "ok"
    assert st.stereo_status_str(1) == "invalid argument"


def test_host_side_argument_checks(L):
    h = C.c_void_p()
    assert L.stereo_create(None, 1, C.byref(h)) == 1
    p = st.stereo_default_params(num_disp=0)
    assert L.stereo_create(C.byref(p), 1, C.byref(h)) == 1
    p = st.stereo_default_params(win_radius=9)
    assert L.stereo_create(C.byref(p), 1, C.byref(h)) == 1
    p = st.stereo_default_params()
    assert L.stereo_create(C.byref(p), 0, C.byref(h)) == 1
    # stage calls validate sizes and pointers before any launch
    assert L.stereo_stage_lr(None, None, 10, 10, 1, None, None) == 1
    assert L.stereo_stage_outlier(None, C.c_void_p(16), 0, 10, 10, 2.5, C.c_void_p(32), None) == 1
    assert L.stereo_stage_fill_disc(None, C.c_void_p(16), 8, 8, 20, -1, C.c_void_p(32), None) == 1
    assert L.stereo_match(None, None, None) == 1
    assert L.stereo_gray(None, 4, 4, 12, None, None) == 1
    cam = st.StereoCamera(500.0, 10.0, 10.0, 5.0, 0.0)
    assert L.stereo_depth_points(None, 8, 8, C.byref(cam), C.c_void_p(16), None, None) == 1
    assert L.stereo_depth_points(C.c_void_p(16), 8, 8, C.byref(cam), None, None, None) == 1   # no output
    bad = st.StereoCamera(0.0, 10.0, 10.0, 5.0, 0.0)
    assert L.stereo_depth_points(C.c_void_p(16), 8, 8, C.byref(bad), C.c_void_p(16), None, None) == 1
    assert L.stereo_vote_nbins(4.0, 128.0) == 64 and L.stereo_vote_nbins(0.0, 1.0) == 0
    assert L.stereo_vote_matches(None, None, 10, 4.0, 128.0, None, None, None, None) == 1
    assert L.stereo_destroy(None) == 0


def test_checked_build_loads_and_exports_everything(L):
    stbuild.build(checked=True)
    with st.checked_library() as LC:
        assert LC.stereo_build_checked() == 1
        missing = [n for n in st.header_functions() if not hasattr(LC, n)]
        assert not missing, missing
    assert L.stereo_build_checked() == 0
    assert L.stereo_debug_check_selftest(None) == 4        # STEREO_ERR_UNSUPPORTED in the normal build


def test_injected_allocation_failure_returns_oom_and_frees(L):
    """The first device allocation of stereo_create fails by injection: the
    call returns STEREO_ERR_OOM and holds nothing (no GPU needed: the
    injected failure comes before any cudaMalloc)."""
    live0 = st.stereo_debug_live_allocations()
    st.stereo_debug_fail_alloc(0)
    h = C.c_void_p()
    p = st.stereo_default_params(max_width=64, max_height=32, num_disp=16)
    assert L.stereo_create(C.byref(p), 1, C.byref(h)) == 3          # STEREO_ERR_OOM
    assert st.stereo_debug_live_allocations() == live0
    assert L.stereo_debug_fail_alloc(-2) == 1
    st.stereo_debug_fail_alloc(-1)
