"""Full-size parity of the whole path against the FP64 oracle, on the seeded
workloads at their own sizes and in the launch configuration the benchmark
times (stereo_match on a side stream: the first call captures a CUDA graph,
the second replays it; the replayed outputs are the ones checked).

Every pixel is compared; nothing is skipped.  The check follows the path
stage by stage (Sec. II-A, II-B, II-C):

  * winner-take-all, left and right views: bit-exact with the oracle's
    winners except where the oracle's best and second-best ZNCC differ by
    less than 1e-5 (FP32 may break such a near-tie either way); sub-pixel
    within 0.01 px wherever the winners agree;
  * left-right check and post-processing: the oracle's stages applied to the
    GPU's own winner maps must give the GPU's maps bit for bit, on every
    pixel (so a near-tie flip upstream cannot hide a mismatch downstream);
  * refinement: the oracle's refinement (ZNCC recomputed in FP64 from the
    images) of the GPU's post-processed map against the GPU's refined map:
    the same invalid pixels, and at most 0.5 % of the valid pixels beyond
    1e-4 relative for an FP32 volume (5 % beyond 0.01 px, median <= 1e-3 px,
    for 16-bit volumes, whose storage rounding can flip a near-tied
    o-update).

The end-to-end difference against the oracle's own whole path (its stages
applied to its own winners) is reported beside these: disparity error
(max |dd|, share of pixels beyond 0.01 px) per workload and cost format.
With STEREO_PARITY_REPORT set, every figure is appended to that file as a
JSON line.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import (NEAR_TIE, SUB_TOL, REFINE_RTOL, to_np, int_map_mismatch, describe,
                    oracle_match_rows, oracle_soft_rows, report)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402

INV = oracle.INVALID
CDT = {"f32": st.COST_F32, "f16": st.COST_F16, "bf16": st.COST_BF16, "none": st.COST_NONE}

# name -> (generator, oracle.Params, cost formats); the sizes are the
# benchmark workloads' sizes
WORKLOADS = {
    "perlin320": (lambda: synth.perlin_pair(synth.seed_for(0)),
                  oracle.Params(d_min=0, num_disp=32, win_radius=5, smooth_radius=2), ("f32",)),
    "tissue960": (lambda: synth.tissue_pair(synth.seed_for(1)),
                  oracle.Params(d_min=0, num_disp=128, win_radius=5, smooth_radius=15), ("f32", "none")),
    "tissue960_d192": (lambda: synth.tissue_pair(synth.seed_for(2), 960, 540, 10.0, 170.0),
                       oracle.Params(d_min=0, num_disp=192, win_radius=7, smooth_radius=15),
                       ("f16", "bf16", "f32")),
    "paper960": (lambda: synth.tissue_pair(synth.seed_for(5), 960, 540, -10.0, 70.0),
                 oracle.Params(d_min=-20, num_disp=100, win_radius=5, smooth_radius=15,
                               sampling=oracle.SAMPLE_CHESSBOARD), ("f32",)),
}


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    st.lib()
    return torch.device("cuda:0")


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _gray(img):
    return img if img.ndim == 2 else oracle.gray(img)


def gpu_whole_path(dev, Limg, Rimg, p: oracle.Params, cdt):
    """stereo_match on a side stream, captured then replayed (as timed by
    the benchmark), plus the right-view winners from the stage entry point
    (the same cost kernel)."""
    H, W = Limg.shape[:2]
    sp = st.stereo_default_params(max_width=W, max_height=H, d_min=p.d_min, num_disp=p.num_disp,
                                  win_radius=p.win_radius, cost_dtype=cdt, sampling=p.sampling,
                                  smooth_radius=p.smooth_radius, smooth_iters=p.smooth_iters)
    h = st.stereo_create(sp)
    tL, tR = T(Limg, dev), T(Rimg, dev)
    out = dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
               disp_sub=torch.empty((H, W), dtype=torch.float32, device=dev),
               disp_lr=torch.empty((H, W), dtype=torch.int16, device=dev),
               disp_post=torch.empty((H, W), dtype=torch.int16, device=dev),
               valid=torch.empty((H, W), dtype=torch.uint8, device=dev),
               disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))
    s = torch.cuda.Stream()
    for _ in range(2):
        for v in out.values():
            v.fill_(7)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            st.stereo_match(h, tL, tR, **out, stream=s)
        s.synchronize()
    g = {k: to_np(v) for k, v in out.items()}
    gl = T(_gray(Limg), dev)
    gr = T(_gray(Rimg), dev)
    dl = torch.empty((H, W), dtype=torch.int16, device=dev)
    dr = torch.empty_like(dl)
    sub = torch.empty((H, W), dtype=torch.float32, device=dev)
    st.stereo_stage_match(h, gl, gr, p.d_min, p.num_disp, p.win_radius, p.sampling,
                          st.COST_NONE if cdt == st.COST_NONE else cdt, dl, dr, sub,
                          None if cdt == st.COST_NONE else
                          torch.empty((H, W, st.cost_stride(p.num_disp)),
                                      dtype={st.COST_F32: torch.float32, st.COST_F16: torch.float16,
                                             st.COST_BF16: torch.bfloat16}[cdt], device=dev))
    torch.cuda.synchronize()
    h.close()
    g["dL"], g["dR"] = to_np(dl), to_np(dr)
    return g


def check_winners(g, m, name):
    """Left and right winners bit-exact outside the oracle's near-ties;
    sub-pixel within 0.01 px where the winners agree.  Returns stats."""
    assert np.array_equal(g["dL"], g["disp_wta"]), "stage entry point and whole path disagree"
    nearL, nearR = m["gapL"] < NEAR_TIE, m["gapR"] < NEAR_TIE
    bad = int_map_mismatch(g["dL"], m["dL"], nearL)
    assert len(bad) == 0, f"{name} left WTA: " + describe(bad, g["dL"], m["dL"], m["gapL"])
    bad = int_map_mismatch(g["dR"], m["dR"], nearR)
    assert len(bad) == 0, f"{name} right WTA: " + describe(bad, g["dR"], m["dR"], m["gapR"])
    same = (g["dL"] == m["dL"]) & (m["dL"] != INV)
    err = np.abs(g["disp_sub"][same] - m["sub"][same])
    assert err.size and err.max() <= SUB_TOL, f"{name} sub-pixel max {err.max():.3e}"
    return dict(pixels=int(g["dL"].size), wta_near_tie_exempt=int(nearL.sum()),
                wta_flipped_near_ties=int((g["dL"] != m["dL"]).sum()),
                right_flipped_near_ties=int((g["dR"] != m["dR"]).sum()),
                subpixel_max_abs=float(err.max()), subpixel_pct_gt_0p01=float(100 * np.mean(err > 0.01)))


def refine_stats(got, ref):
    nan_g, nan_r = np.isnan(got), np.isnan(ref)
    assert np.array_equal(nan_g, nan_r), "refined maps differ in their invalid pixels"
    v = ~nan_r
    d = np.abs(got[v] - ref[v])
    rel = d / np.maximum(np.abs(ref[v]), 1)
    return d, rel, dict(valid=int(v.sum()), max_abs=float(d.max(initial=0)),
                        pct_gt_0p01=float(100 * np.mean(d > 0.01)) if d.size else 0.0,
                        pct_rel_gt_1e4=float(100 * np.mean(rel > REFINE_RTOL)) if d.size else 0.0,
                        median_abs=float(np.median(d)) if d.size else 0.0)


_REFINE_MEMO = {}


def oracle_refine(o_post, Lg, Rg, p):
    """oracle.refine with the ZNCC recomputed from the images, memoised on
    its inputs (the cost formats of one workload usually share them)."""
    import hashlib
    key = hashlib.sha1(o_post.tobytes() + Lg.tobytes() + Rg.tobytes() + repr(p).encode()).hexdigest()
    if key not in _REFINE_MEMO:
        _REFINE_MEMO[key] = oracle.refine(o_post, None, Lg, Rg, p)[0]
    return _REFINE_MEMO[key]


def check_chain(g, Lg, Rg, p, fmt, name):
    """The oracle's LR check and post-processing on the GPU's own winners
    reproduce the GPU maps bit for bit; its refinement matches within the
    refinement bar."""
    o_lr = oracle.lr_check(g["dL"], g["dR"], p.lr_thresh)
    bad = int_map_mismatch(g["disp_lr"], o_lr)
    assert len(bad) == 0, f"{name} LR check: " + describe(bad, g["disp_lr"], o_lr)
    o_post = oracle.postprocess(o_lr, p)
    bad = int_map_mismatch(g["disp_post"], o_post)
    assert len(bad) == 0, f"{name} post-processing: " + describe(bad, g["disp_post"], o_post)
    assert np.array_equal(g["valid"].astype(bool), o_post != INV)
    d_ref = oracle_refine(o_post, Lg, Rg, p)
    d, rel, stats = refine_stats(g["disp_final"], d_ref)
    if fmt in ("f32", "none"):
        assert np.mean(rel > REFINE_RTOL) <= 0.005, stats
    else:
        assert np.mean(d > 0.01) <= 0.05 and np.median(d) <= 1e-3, stats
    return o_post, stats


def end_to_end_stats(g, m, Lg, Rg, p):
    """The GPU whole path against the oracle's own whole path (its stages on
    its own winners).  Identical to the chain when no near-tie flipped."""
    o_post = oracle.postprocess(oracle.lr_check(m["dL"], m["dR"], p.lr_thresh), p)
    d_ref = oracle_refine(o_post, Lg, Rg, p)
    post_diff = float(100 * np.mean(g["disp_post"] != o_post))
    both = ~np.isnan(d_ref) & ~np.isnan(g["disp_final"])
    d = np.abs(g["disp_final"][both] - d_ref[both])
    return dict(e2e_post_pct_differ=post_diff,
                e2e_valid_pct_differ=float(100 * np.mean(np.isnan(d_ref) != np.isnan(g["disp_final"]))),
                e2e_final_max_abs=float(d.max(initial=0)),
                e2e_final_pct_gt_0p01=float(100 * np.mean(d > 0.01)) if d.size else 0.0)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_whole_path_full_size(dev, name):
    gen, p, fmts = WORKLOADS[name]
    pair = gen()
    Limg, Rimg = pair[0], pair[1]
    Lg, Rg = _gray(Limg), _gray(Rimg)
    H, W = Lg.shape
    m = oracle_match_rows(Lg, Rg, p.d_min, p.num_disp, p.win_radius, p.sampling)
    for fmt in fmts:
        g = gpu_whole_path(dev, Limg, Rimg, p, CDT[fmt])
        wstats = check_winners(g, m, f"{name}/{fmt}")
        o_post, rstats = check_chain(g, Lg, Rg, p, fmt, f"{name}/{fmt}")
        estats = end_to_end_stats(g, m, Lg, Rg, p)
        report(name, cost=fmt, size=f"{W}x{H}", d_min=p.d_min, num_disp=p.num_disp,
               window=2 * p.win_radius + 1, sampling="chessboard" if p.sampling else "full", **wstats,
               lr_post_chain="bit-exact", **{"refine_" + k: v for k, v in rstats.items()}, **estats)


# ------------------------------------------------------------------ batched form
BATCH_PICK = (3, 17, 39, 56)     # 640x480 D192 r7, 960x540 D128 r5, 1280x720 D64 r7, 1920x1080 D192 r7
STRIP_1080 = (500, 564)          # rows of the 1920x1080 pair compared with the oracle


def test_batched_size_classes_full_size(dev):
    """One pair of each size class of the 64-pair workload, run together as
    one batch (persistent cost launch, graph-replayed, FP16 volume): every
    output of every pair bit-identical to the single-pair path; the winners
    of the three smaller pairs on every pixel, and of the 1920x1080 pair on
    a 64-row strip, against the oracle (near-ties exempt)."""
    specs = [synth.batch_pair(i) for i in BATCH_PICK]
    maxW = max(s[3]["W"] for s in specs)
    maxH = max(s[3]["H"] for s in specs)
    maxD = max(s[3]["D"] for s in specs)
    p = st.stereo_default_params(max_width=maxW, max_height=maxH, num_disp=maxD, win_radius=7,
                                 cost_dtype=st.COST_F16, smooth_radius=15)
    hb = st.stereo_create(p, max_batch=len(specs))
    batch = []
    for L, R, gt, sp in specs:
        H, W = sp["H"], sp["W"]
        batch.append(dict(left=T(L, dev), right=T(R, dev), d_min=0, num_disp=sp["D"], win_radius=sp["r"],
                          disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                          disp_sub=torch.empty((H, W), dtype=torch.float32, device=dev),
                          disp_post=torch.empty((H, W), dtype=torch.int16, device=dev),
                          disp_final=torch.empty((H, W), dtype=torch.float32, device=dev)))
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(2):                            # capture, then replay
        with torch.cuda.stream(s):
            st.stereo_match_batched(hb, batch, use_graph=True, stream=s)
        s.synchronize()
    # the other stage mode (one launch per stage over all pairs) gives the same maps
    st.stereo_set_batch_stages(hb, 1)
    keys = ("disp_wta", "disp_sub", "disp_post", "disp_final")
    other = [dict(b, **{k: torch.empty_like(b[k]) for k in keys}) for b in batch]
    for _ in range(2):
        with torch.cuda.stream(s):
            st.stereo_match_batched(hb, other, use_graph=True, stream=s)
        s.synchronize()
    for b, o in zip(batch, other):
        for k in keys:
            assert torch.equal(b[k].nan_to_num(-7), o[k].nan_to_num(-7)), k
    hb.close()
    for (L, R, gt, sp), b in zip(specs, batch):
        H, W, D, r = sp["H"], sp["W"], sp["D"], sp["r"]
        ps = st.stereo_default_params(max_width=W, max_height=H, num_disp=D, win_radius=r,
                                      cost_dtype=st.COST_F16, smooth_radius=15)
        hs = st.stereo_create(ps)
        one = {k: torch.empty_like(b[k]) for k in ("disp_wta", "disp_sub", "disp_post", "disp_final")}
        st.stereo_match(hs, b["left"], b["right"], **one)
        torch.cuda.synchronize()
        hs.close()
        for k in one:
            assert torch.equal(one[k].nan_to_num(-1), b[k].nan_to_num(-1)), (sp, k)
        Lg, Rg = oracle.gray(L), oracle.gray(R)
        y0, y1 = (0, H) if H < 1080 else STRIP_1080
        m = oracle_match_rows(Lg, Rg, 0, D, r, 0, y0, y1)
        got = to_np(b["disp_wta"])[y0:y1]
        sub = to_np(b["disp_sub"])[y0:y1]
        near = m["gapL"] < NEAR_TIE
        bad = int_map_mismatch(got, m["dL"], near)
        assert len(bad) == 0, describe(bad, got, m["dL"], m["gapL"])
        same = (got == m["dL"]) & (m["dL"] != INV)
        err = np.abs(sub[same] - m["sub"][same])
        assert err.max() <= SUB_TOL
        report(f"batch64/{W}x{H}/D{D}/r{r}", cost="f16", rows_compared=f"{y0}..{y1 - 1}",
               pixels=int(got.size), wta_near_tie_exempt=int(near.sum()),
               wta_flipped_near_ties=int((got != m["dL"]).sum()), subpixel_max_abs=float(err.max()),
               subpixel_pct_gt_0p01=float(100 * np.mean(err > 0.01)),
               downstream="bit-identical to the single-pair path")


# ------------------------------------------------------------------ soft-argmin form
SOFT_STRIP = (200, 232)


def test_soft_argmin_full_size_strip(dev):
    """Two 960x540 pairs of the differentiation workload (D = 128, r = 5,
    tau = 0.1), forward and backward over the whole images with a random
    upstream gradient; on a 32-row strip of each the oracle's d_soft
    (within 1e-4 px) and image gradients (relative L2 <= 1e-3)."""
    B, H, W, D, r, tau = 2, 540, 960, 128, 5, 0.1
    pairs = [synth.tissue_pair(synth.seed_for(4, b)) for b in range(B)]
    L = np.stack([oracle.gray(q[0]) for q in pairs]).astype(np.float32)
    R = np.stack([oracle.gray(q[1]) for q in pairs]).astype(np.float32)
    h = st.stereo_create(st.stereo_default_params(max_width=W, max_height=H, num_disp=D, soft_argmin=1))
    tL, tR = T(L, dev), T(R, dev)
    ds = torch.empty((B, H, W), dtype=torch.float32, device=dev)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, tL, tR, 0, D, r, tau, ds, lse)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    g = np.where(np.isnan(to_np(ds)), 0.0, rng.normal(0, 1, (B, H, W))).astype(np.float32)
    gL, gR = torch.empty_like(ds), torch.empty_like(ds)
    st.stereo_softargmin_bwd(h, tL, tR, 0, D, r, tau, ds, lse, T(g, dev), gL, gR)
    torch.cuda.synchronize()
    h.close()
    y0, y1 = SOFT_STRIP
    for b in range(B):
        o = oracle_soft_rows(L[b], R[b], 0, D, r, tau, g[b], y0, y1)
        got = to_np(ds[b])[y0:y1]
        assert np.array_equal(np.isnan(got), ~o["hv"])
        dmax = float(np.max(np.abs(got[o["hv"]] - o["ds"][o["hv"]])))
        assert dmax <= 1e-4
        rels = []
        for gg, ref in ((to_np(gL[b])[y0:y1], o["gL"]), (to_np(gR[b])[y0:y1], o["gR"])):
            rel = float(np.linalg.norm(gg - ref) / np.linalg.norm(ref))
            rels.append((rel, float(np.max(np.abs(gg - ref)))))
            assert rel <= 1e-3
        report("soft8", pair=b, size=f"{W}x{H}", rows_compared=f"{y0}..{y1 - 1}", num_disp=D, tau=tau,
               d_soft_max_abs=dmax, d_soft_pct_gt_0p01=float(100 * np.mean(np.abs(got[o["hv"]] - o["ds"][o["hv"]]) > 0.01)),
               gradL_rel_l2=rels[0][0], gradL_max_abs=rels[0][1], gradR_rel_l2=rels[1][0], gradR_max_abs=rels[1][1])
