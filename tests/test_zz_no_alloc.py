"""The allocation-free entry point, stereo_match_wta_noalloc.

It exists for callers that must not allocate device memory while matching
(for example a real-time video pipeline that forbids allocation after
start-up, or a host that lends a plugin only its image and output buffers):
the scratch lives in a fixed array inside the library.  These tests call it
through the C ABI and check it against stereo_stage_match (same stage, handle
workspace, no cost volume) on two calls in a row.  The file is named to be
collected last, and it needs no state from earlier tests.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402


def _via_abi(tL, tR, d_min, D, r, stream):
    H, W = tL.shape
    dl = torch.full((H, W), 7, dtype=torch.int16, device=tL.device)
    dr = torch.full((H, W), 7, dtype=torch.int16, device=tL.device)
    sub = torch.full((H, W), 7.0, dtype=torch.float32, device=tL.device)
    status = st.lib().stereo_match_wta_noalloc(
        C.c_void_p(tL.data_ptr()), C.c_void_p(tR.data_ptr()), W, H, d_min, D, r,
        C.c_void_p(dl.data_ptr()), C.c_void_p(dr.data_ptr()), C.c_void_p(sub.data_ptr()),
        C.c_void_p(stream.cuda_stream))
    assert status == 0, st.stereo_status_str(status)
    return dl, dr, sub


def _with_handle(tL, tR, d_min, D, r):
    H, W = tL.shape
    p = st.stereo_default_params(max_width=W, max_height=H, num_disp=D, d_min=d_min, win_radius=r,
                                 cost_dtype=st.COST_NONE)
    h = st.stereo_create(p)
    dl = torch.empty((H, W), dtype=torch.int16, device=tL.device)
    dr = torch.empty_like(dl)
    sub = torch.empty((H, W), dtype=torch.float32, device=tL.device)
    st.stereo_stage_match(h, tL, tR, d_min, D, r, st.SAMPLE_FULL, st.COST_NONE, dl, dr, sub, None)
    torch.cuda.synchronize()
    h.close()
    return dl, dr, sub


@pytest.mark.parametrize("case,d_min", [("perlin320", 0), ("tissue640", -4),
                                        ("tissue640", 64), ("tissue640", -64)])
def test_noalloc_matches_stage_match_twice(case, d_min):
    """The 640x480 cases are the largest size the fixed scratch accepts, with
    D = 128 and r = 7; d_min = +64 and -64 are the extremes of the accepted
    range, which put the staged rows' column offsets at their largest."""
    assert torch.cuda.is_available()
    dev = torch.device("cuda:0")
    if case == "perlin320":
        L, R, _ = synth.perlin_pair(synth.seed_for(0))
        D, r = 32, 5
    else:
        Lrgb, Rrgb, _ = synth.tissue_pair(synth.seed_for(1), 640, 480)
        w = np.array([77, 150, 29])
        L = ((Lrgb.astype(np.int32) @ w + 128) >> 8).astype(np.uint8)
        R = ((Rrgb.astype(np.int32) @ w + 128) >> 8).astype(np.uint8)
        D, r = 128, 7
    tL = torch.from_numpy(np.ascontiguousarray(L)).to(dev)
    tR = torch.from_numpy(np.ascontiguousarray(R)).to(dev)
    want = _with_handle(tL, tR, d_min, D, r)
    s = torch.cuda.Stream()
    for _ in range(2):                     # the second call reuses the same scratch
        got = _via_abi(tL, tR, d_min, D, r, s)
        s.synchronize()
        assert torch.equal(got[0], want[0])
        assert torch.equal(got[1], want[1])
        a, b = got[2].cpu().numpy(), want[2].cpu().numpy()
        assert np.array_equal(np.isnan(a), np.isnan(b))
        ok = ~np.isnan(b)
        assert np.max(np.abs(a[ok] - b[ok]), initial=0.0) <= 0.01


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dev = torch.device("cuda:0")
    t = torch.zeros((481, 640), dtype=torch.uint8, device=dev)
    o = torch.zeros((481, 640), dtype=torch.int16, device=dev)
    L = st.lib()
    args = lambda W, H, dmin, D: (C.c_void_p(t.data_ptr()), C.c_void_p(t.data_ptr()), W, H, dmin, D, 5,
                                  C.c_void_p(o.data_ptr()), C.c_void_p(o.data_ptr()), None, None)
    assert L.stereo_match_wta_noalloc(*args(640, 481, 0, 64)) == 6      # STEREO_ERR_TOO_LARGE
    assert L.stereo_match_wta_noalloc(*args(641, 100, 0, 64)) == 6
    assert L.stereo_match_wta_noalloc(*args(320, 240, 0, 129)) == 6
    assert L.stereo_match_wta_noalloc(*args(320, 240, 65, 32)) == 6
    assert L.stereo_match_wta_noalloc(*args(320, 240, 0, 0)) == 1       # STEREO_ERR_INVALID_ARG
