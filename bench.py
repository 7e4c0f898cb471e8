#!/usr/bin/env python
"""Benchmark of the dense stereo-matching path (arXiv 2007.12623, Sec. II) on
B300.

Default workload (``tissue960``): one step = the whole path on one 960x540 RGB
tissue pair (D = 128, 11x11 ZNCC window, FP32 cost volume, LR check, 3
outlier/hole-filling rounds, 5 refinement iterations with radius 15): gray ->
window statistics -> fused ZNCC + winner-take-all (left and right) + cost
store -> sub-pixel / LR -> outlier + hole filling -> improved Laplacian
refinement.

Other workloads (``--workload``):
  tissue960_d192_f16 / _bf16  same generator, D = 192, 15x15 window, cost
                              volume stored in FP16 / BF16 (their disparity
                              error against the FP64 oracle is measured by
                              tests/test_gpu_precision.py).
  tissue960_x4 / _x4_f16      4 pairs of the default workload's generator per
                              stereo_match_batched call (a stream of pairs
                              matched 4 at a time), FP32 / FP16 volume.
  batch64                     64 pairs of mixed sizes (16 each of 640x480,
                              960x540, 1280x720, 1920x1080), D in {64,128,192},
                              windows {9,11,15}, FP16 cost: one
                              stereo_match_batched call per step (one
                              persistent cost launch, graph-replayed),
                              configuration from the autotuner.
  soft8                       soft-argmin form: 8 pairs at 960x540, D = 128,
                              11x11, tau = 0.1; a step is forward + L1 loss +
                              hand-written backward to both images through
                              torch.autograd.
  paper960                    the paper's own setting: chessboard-sampled 11x11
                              window, d in [-20, 80), smoothing radius 15.
  perlin320                   the small 320x240 gray Perlin pair (D = 32).

With no ``--workload`` the line also carries a ``workloads`` record of every
other workload, each measured by ``bench.py --workload NAME`` in a process of
its own.

Prints one JSON line (rank 0).  ``value`` is pixel-disparity evaluations per
second of the whole step (Gpix*disp/s) with inputs resident in device memory;
``e2e`` is the same metric through the public API with the inputs copied from
pinned host memory and the result copied back inside the timed region.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload instead.

Multi-GPU: one process per GPU (torchrun); every rank matches its own pairs
(independent problems, no collective), ``scaling`` is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOADS = {
    # 960x540 RGB tissue pair, D = 0..127, 11x11 window, FP32 cost, full post-processing
    "tissue960": dict(kind="single", W=960, H=540, D=128, r=5, cost="f32", smooth_radius=15,
                      seed=synth.seed_for(1), disp=(10.0, 110.0)),
    # 960x540, D = 0..191, 15x15 window, FP16 / BF16 cost storage
    "tissue960_d192_f16": dict(kind="single", W=960, H=540, D=192, r=7, cost="f16", smooth_radius=15,
                               seed=synth.seed_for(2), disp=(10.0, 170.0)),
    "tissue960_d192_bf16": dict(kind="single", W=960, H=540, D=192, r=7, cost="bf16", smooth_radius=15,
                                seed=synth.seed_for(2), disp=(10.0, 170.0)),
    # same-workload comparisons: the 960x540 D = 128 pair with an FP16 volume
    # and without a volume; the D = 192 pair with an FP32 volume
    "tissue960_f16": dict(kind="single", W=960, H=540, D=128, r=5, cost="f16", smooth_radius=15,
                          seed=synth.seed_for(1), disp=(10.0, 110.0)),
    "tissue960_none": dict(kind="single", W=960, H=540, D=128, r=5, cost="none", smooth_radius=15,
                           seed=synth.seed_for(1), disp=(10.0, 110.0)),
    "tissue960_d192_f32": dict(kind="single", W=960, H=540, D=192, r=7, cost="f32", smooth_radius=15,
                               seed=synth.seed_for(2), disp=(10.0, 170.0)),
    # 64 mixed pairs in one batched call, FP16 cost
    "batch64": dict(kind="batched", n=64, cost="f16", smooth_radius=15),
    # a stream of 960x540 D = 128 pairs matched 4 at a time through the
    # batched call (throughput form of the single-pair workload), FP32 / FP16
    "tissue960_x4": dict(kind="batched", n=4, cost="f32", smooth_radius=15, same="tissue960"),
    "tissue960_x4_f16": dict(kind="batched", n=4, cost="f16", smooth_radius=15, same="tissue960"),
    # one pair of each size class of the 64-pair batch (a small batched case
    # for profiling): 640x480 D192 r7, 960x540 D128 r5, 1280x720 D64 r7,
    # 1920x1080 D192 r7
    "batch4": dict(kind="batched", n=4, cost="f16", smooth_radius=15, pick=(3, 17, 39, 56)),
    # soft-argmin training step on 8 pairs
    "soft8": dict(kind="soft", B=8, W=960, H=540, D=128, r=5, tau=0.1, seed=synth.seed_for(4),
                  disp=(10.0, 110.0)),
    # the paper's own configuration: chessboard-sampled 11x11 window, candidates
    # d in [-20, 80), smoothing radius 15, 960x540 tissue pair (field -10..70)
    "paper960": dict(kind="single", W=960, H=540, D=100, d_min=-20, r=5, cost="f32", smooth_radius=15,
                     sampling=1, seed=synth.seed_for(5), disp=(-10.0, 70.0)),
    # 320x240 gray Perlin pair, D = 0..31, 5x5 smoothing
    "perlin320": dict(kind="single", W=320, H=240, D=32, r=5, cost="f32", smooth_radius=2,
                      seed=synth.seed_for(0), disp=None),
}
COST_CODE = {"none": 0, "f32": 1, "f16": 2, "bf16": 3}
# DRAM bytes (read + write) of one launch of the workload's dominant kernel,
# read from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of
# the kernel as it is built now; absent where no such capture exists.
KERNEL_TRAFFIC = {"tissue960": 222.2e6, "tissue960_f16": 94.4e6, "tissue960_none": 18.6e6,
                  # one persistent launch over the 4 pairs
                  "tissue960_x4": 1062.8e6, "tissue960_x4_f16": 547.3e6,
                  # both launches of the D = 192 range (128 at K = 4, 64 at K = 2)
                  "tissue960_d192_f16": 130.0e6,
                  "soft8": {"k_soft_box_t1": 606.8e6, "k_cost_wta (soft backward form)": 235.5e6}}
COST_BYTES = {"none": 0, "f32": 4, "f16": 2, "bf16": 2}
METRIC = "Gpix*disp/s and ms per 960x540 pair (1 B300), % of roofline, vs oracle"
DATA = "synthetic (seeded tissue-texture generator standing in for the paper's videos)"
UNIT = "Gpix*disp/s"
L2_BYTES = 126 * 2 ** 20
L2_NOTE = ("flushed between timed steps on the step's stream (252 MiB write, then a 126 MiB read "
           "that leaves no dirty line of the flush; untimed)")
PAPER_CONTEXT = {"ms_per_keyframe_whole_pipeline": 76.3, "stereo_stage_ms": 15.9,
                 "zncc_ms_960x540x100": 5.0,
                 "hardware": "NVIDIA Titan X + Xeon X5472 (paper, Table III)"}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), sm_max_mhz=float(p.get("sm_max_mhz", 2032.0)),
                    source="measured")
    except Exception:
        return dict(hbm_gbs=6400.0, sm_max_mhz=2032.0, source="fallback")


def rank_pair_ids(wl, rank):
    """The pairs rank `rank` matches (replicas share nothing): single-pair
    workloads take generator pair `rank`, batched ones pairs rank * n ..
    rank * n + n - 1 of their generator (or the picked pairs), the
    soft-argmin step pairs rank * B .. rank * B + B - 1."""
    if wl["kind"] == "batched":
        if wl.get("pick"):
            return [p + 64 * rank for p in wl["pick"]]
        return list(range(rank * wl["n"], rank * wl["n"] + wl["n"]))
    if wl["kind"] == "soft":
        return list(range(rank * wl["B"], rank * wl["B"] + wl["B"]))
    return [rank]


def make_pair(wl, pair_index=0):
    if wl["disp"] is None:
        L, R, gt = synth.perlin_pair(wl["seed"] + pair_index, wl["W"], wl["H"])
        return np.stack([L] * 3, -1), np.stack([R] * 3, -1), gt
    return synth.tissue_pair(wl["seed"] + pair_index, wl["W"], wl["H"], *wl["disp"])


def _batch_pair(i):
    return synth.batch_pair(i)


def _same_pair(args):
    name, i = args
    wl = WORKLOADS[name]
    L, R, gt = make_pair(wl, i)
    return L, R, gt, dict(W=wl["W"], H=wl["H"], D=wl["D"], r=wl["r"])


def make_batch(ids, same=None):
    """Pairs `ids` of the mixed batch's generator (or, with `same`, of that
    single-pair workload's generator), generated by a spawn pool (started
    before any CUDA call)."""
    import multiprocessing as mp
    procs = max(1, min(len(ids), os.cpu_count() or 1, 32))
    with mp.get_context("spawn").Pool(procs) as pool:
        if same:
            return pool.map(_same_pair, [(same, i) for i in ids])
        return pool.map(_batch_pair, ids)


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first_sample(self, busy, timeout=5.0):
        """Runs `busy()` until the sampler has produced a line (or timeout)."""
        t0 = time.time()
        n0 = len(self.lines)
        while self.proc and len(self.lines) <= n0 and time.time() - t0 < timeout:
            for _ in range(5):
                busy()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- roofline

def cost_kernel_roofline(problems, cost_ms, peaks, sm_count, kernel, traffic=None):
    """Roofline of the fused cost + winner-take-all kernel over `problems`
    (list of (W, H, D, r, cost storage)) done by one launch.

    Algorithmic work per pixel-disparity (p,d) with a full window: 12 FP32/INT32
    issue slots (1 product, 2 vertical + 2 horizontal sliding-sum updates, 2
    for the numerator, 2 for rho, 2 for the winner compare/select, 1 for the
    store conversion) and s bytes of cost store (s = 4 FP32, 2 FP16/BF16).  Per
    pixel it also reads both gray images (2 B), both statistics maps (16 B) and
    writes both key maps (8 B).  The bound is whichever of the ALU time (12 ops
    on 128 lanes per SM per clock) and the HBM time is longer.
    """
    bytes_, ops = 0, 0
    for W, H, D, r, cost in problems:
        P = (W - 2 * r) * (H - 2 * r) * D
        bytes_ += P * COST_BYTES[cost] + W * H * (2 + 16 + 8)
        ops += 12 * P
    t_hbm = bytes_ / (peaks["hbm_gbs"] * 1e9)
    alu_peak = sm_count * 128 * peaks["sm_max_mhz"] * 1e6          # ops/s at max clock
    t_alu = ops / alu_peak
    dur = cost_ms * 1e-3
    if t_hbm >= t_alu:
        achieved = bytes_ / dur / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "kernel": kernel, "algorithmic_bytes": bytes_, "algorithmic_ops": ops,
                "kernel_ms": round(cost_ms, 4), "peak_source": peaks["source"] + " (hbm_gbs)"}
    achieved = ops / dur / 1e12
    return {"bound": "alu", "achieved": round(achieved, 2), "peak": round(alu_peak / 1e12, 2),
            "unit": "Tops/s", "frac": round(achieved / (alu_peak / 1e12), 4), "traffic": traffic,
            "kernel": kernel, "algorithmic_ops": ops, "algorithmic_bytes": bytes_,
            "kernel_ms": round(cost_ms, 4),
            "peak_source": f"{sm_count} SMs x 128 lanes x {peaks['sm_max_mhz']:.0f} MHz"}


def soft_roofline(stage_ms, W, H, D, peaks, sm_count, traffic=None):
    """Roofline of the dominant soft-argmin backward kernel.
      cost kernel, backward form (D <= 128, stage "cost"): per (p,d) 25
                     FP32 issue slots (9 for the ZNCC as in the cost kernel's
                     count without the winner, 16 for the backward terms: the
                     exponent and its argument, G, A, the two P and two Q
                     terms) and the A store (4 B); per pixel it reads both
                     images, both statistics maps, g, d_soft and lse and
                     writes P1, P2 and adds into Q1, Q2 (60 B).  The bound is
                     whichever of the ALU time (128 lanes per SM per clock)
                     and the HBM time is longer.
      k_soft_dA      (D > 128, stage "dA") reads the FP32 cost volume and
                     writes the A volume (8 B per (p,d)), per pixel reads g,
                     d_soft, lse and the left statistics (20 B) and writes
                     P1, P2, Q1, Q2 (16 B);
      k_soft_box_t1  reads the A volume once (4 B per (p,d)), per pixel reads
                     both images (8 B) and adds into T1L, T1R (8 B)."""
    P, npix = W * H * D, W * H
    fused = D <= 128
    first = ("k_cost_wta (soft backward form)", stage_ms["cost"], 4 * P + 60 * npix, 25 * P) if fused else \
        ("k_soft_dA", stage_ms["dA"], 8 * P + 36 * npix, 0)
    second = ("k_soft_box_t1", stage_ms["box_t1"], 4 * P + 16 * npix, 0)
    name, ms, b, ops = first if first[1] >= second[1] else second
    if isinstance(traffic, dict):
        traffic = traffic.get(name)
    dur = ms * 1e-3
    alu_peak = sm_count * 128 * peaks["sm_max_mhz"] * 1e6
    if ops and ops / alu_peak > b / (peaks["hbm_gbs"] * 1e9):
        achieved = ops / dur / 1e12
        return {"bound": "alu", "achieved": round(achieved, 2), "peak": round(alu_peak / 1e12, 2),
                "unit": "Tops/s", "frac": round(achieved / (alu_peak / 1e12), 4), "traffic": traffic,
                "kernel": name, "algorithmic_ops": ops, "algorithmic_bytes": b, "kernel_ms": round(ms, 4),
                "peak_source": f"{sm_count} SMs x 128 lanes x {peaks['sm_max_mhz']:.0f} MHz"}
    achieved = b / dur / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic, "kernel": name,
            "algorithmic_bytes": b, "algorithmic_ops": ops, "kernel_ms": round(ms, 4),
            "peak_source": peaks["source"] + " (hbm_gbs)"}


# ------------------------------------------------------------- helpers

def _flush_l2(stream, flush, i):
    """Evicts the previous step's data from L2 before the next timed step, on
    the step's own stream (a flush on another stream would run alongside the
    step): a write of a buffer twice the size of L2, then a read of its first
    half, which was evicted first, so that the write's dirty lines are written
    back here and not during the step's first kernels."""
    import torch
    with torch.cuda.stream(stream):
        flush.fill_(float(i))
        flush[: flush.numel() // 2].sum()


def _timed_loop(torch, stream, steps, step, flush):
    """Times `steps` calls of step() on `stream` with CUDA events, flushing L2
    (untimed) before each; returns per-step ms."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        _flush_l2(stream, flush, i)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def _max_over_ranks(torch, dev, x, world):
    """The largest x over all ranks (the slowest rank's time)."""
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _stage_pass(st, h, n, flush, step, names, stream):
    st.stereo_set_stage_timing(h, True)
    acc = {k: 0.0 for k in names}
    for i in range(n):
        _flush_l2(stream, flush, i)
        step()
        ms = st.stereo_get_stage_times(h)
        for k, v in zip(names, ms.values()):
            acc[k] += v
    st.stereo_set_stage_timing(h, False)
    return {k: v / n for k, v in acc.items()}


def _base_line(args, world, value, t_max, dtype, config):
    return {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_max * 1e3 / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": DATA,
            "config": config}


# ------------------------------------------------------------- our arm: one pair

def single_config(name, wl, world):
    """The `config` of a single-pair workload's line (both arms)."""
    return {
        "workload": name, "width": wl["W"], "height": wl["H"], "num_disp": wl["D"], "d_min": wl.get("d_min", 0),
        "window": 2 * wl["r"] + 1, "sampling": "chessboard" if wl.get("sampling", 0) else "full",
        "cost_storage": wl["cost"], "smooth_radius": wl["smooth_radius"], "refine_iters": 5,
        "pairs_per_gpu": 1, "parallelism": f"replicas x{world} (independent pairs)",
        "l2": L2_NOTE,
        "launch": "CUDA graph replay on a non-default stream"}


def run_single(args, wl, rank, world, dev, extras=True):
    import torch
    import paper_2007_12623_b300 as st

    W, H, D = wl["W"], wl["H"], wl["D"]
    Lrgb, Rrgb, gt = make_pair(wl, rank_pair_ids(wl, rank)[0])
    stream = torch.cuda.Stream(dev)          # non-default stream: graph capture + replay
    torch.cuda.set_stream(stream)
    tL = torch.from_numpy(Lrgb).to(dev)
    tR = torch.from_numpy(Rrgb).to(dev)
    sp = st.stereo_default_params(max_width=W, max_height=H, num_disp=D, win_radius=wl["r"],
                                  d_min=wl.get("d_min", 0), sampling=wl.get("sampling", 0),
                                  cost_dtype=COST_CODE[wl["cost"]], smooth_radius=wl["smooth_radius"])
    h = st.stereo_create(sp)
    outs = dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                disp_sub=torch.empty((H, W), dtype=torch.float32, device=dev),
                valid=torch.empty((H, W), dtype=torch.uint8, device=dev),
                disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        st.stereo_match(h, tL, tR, **outs, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        clk.wait_first_sample(step)          # keep the GPU busy until sampling starts
        torch.cuda.synchronize()
        launches0 = st.stereo_launch_count()
        step_ms = _timed_loop(torch, stream, args.steps, step, flush)
    launches = st.stereo_launch_count() - launches0
    t_max = _max_over_ranks(torch, dev, sum(step_ms) / 1e3, world)
    P = W * H * D
    value = world * args.steps * P / t_max / 1e9

    stage_ms = _stage_pass(st, h, min(args.steps, 20), flush, step, st.STAGE_NAMES, stream)
    if extras:
        depth_ms, mosaic_ms, model_points, vote_ms = _single_extras(st, torch, dev, stream, h, W, H, Lrgb,
                                                                     outs, args, flush)
    e2e_value, te = _single_e2e(st, torch, dev, stream, h, Lrgb, Rrgb, tL, tR, W, H, args, world, P)
    h.close()
    if rank != 0:
        return None
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = cost_kernel_roofline([(W, H, D, wl["r"], wl["cost"])], stage_ms["cost_wta"], peaks, sm_count,
                                "k_cost_wta", KERNEL_TRAFFIC.get(args.workload))
    line = _base_line(args, world, value, t_max, "f32", single_config(args.workload, wl, world))
    line.update({
        "ms_per_pair": round(t_max * 1e3 / args.steps, 4),
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "stage_gbs": stage_bandwidth(stage_ms, W, H, D, wl),
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "ms_per_pair": round(te * 1e3 / args.steps, 4),
                "h2d_bytes_per_step": 2 * W * H * 3, "d2h_bytes_per_step": W * H * 4,
                "mode": "stream of pairs: upload of the next and read-back of the previous pair overlap "
                        "the current match (two buffer sets); no L2 flush"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "paper_context": PAPER_CONTEXT,
    })
    if extras:
        line.update({
            "depth_points": _depth_line(W, H, depth_ms, load_peaks()),
            "mosaic_frame": {"ms_median": round(mosaic_ms, 4), "model_points": model_points,
                             "frame_pixels": W * H,
                             "note": "point-based TSDF merge of the refined map's points into the model; "
                                     "event-timed, L2 flushed; not part of the step"},
            "vote_matches": {"ms_median": round(vote_ms, 4), "matches": 2000,
                             "note": "histogram-voting inlier preselection, 85 % outliers; not part of the step"},
        })
    return line


def _single_extras(st, torch, dev, stream, h, W, H, Lrgb, outs, args, flush):
    """Depth, mosaicking and histogram voting on the pair's refined map, each
    event-timed on its own (not part of the step)."""
    # the refined map to points and normals (Sec. II depth from disparity;
    # not part of the step): its own event-timed runs, L2 flushed between
    cam = st.StereoCamera(0.9 * W, W / 2 - 0.5, H / 2 - 0.5, 5.0, 0.0)
    xyz = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    nrm = torch.empty_like(xyz)
    depth_ms = _timed_loop(torch, stream, min(args.steps, 50),
                           lambda: st.stereo_depth_points(outs["disp_final"], cam, xyz, nrm, stream=stream), flush)
    depth_ms = sorted(depth_ms)[len(depth_ms) // 2]

    # point-based TSDF mosaicking of the frame's points into a growing model
    # (Sec. II): 4 warm frames from alternating poses, then timed frames
    img = torch.from_numpy(np.ascontiguousarray(Lrgb)).to(dev)
    model = st.PointModel(8 * W * H, dev)
    poses = []
    for a in (0.0, 0.01):
        c, s_ = np.cos(a), np.sin(a)
        poses.append((np.array([[c, 0, s_], [0, 1, 0], [-s_, 0, c]], np.float32),
                      np.array([0.2 * a * 100, 0.0, 0.0], np.float32)))
    for i in range(4):
        st.stereo_mosaic_frame(h, model, xyz, img, cam, *poses[i % 2], tau=0.5, stream=stream)
    mosaic_ms = _timed_loop(torch, stream, min(args.steps, 20),
                            lambda: st.stereo_mosaic_frame(h, model, xyz, img, cam, *poses[0], tau=0.5,
                                                           stream=stream), flush)
    mosaic_ms = sorted(mosaic_ms)[len(mosaic_ms) // 2]
    model_points = int(model.count.item())

    # histogram-voting preselection of 2000 feature matches (85 % outliers)
    uv1, uv2, _ = synth.feature_matches(synth.seed_for(7), n=2000, inlier_frac=0.15)
    tuv1, tuv2 = torch.from_numpy(uv1).to(dev), torch.from_numpy(uv2).to(dev)
    vh, vs, vo = st.stereo_vote_matches(tuv1, tuv2, stream=stream)
    vote_ms = _timed_loop(torch, stream, min(args.steps, 20),
                          lambda: st.stereo_vote_matches(tuv1, tuv2, hist=vh, score=vs, order=vo, stream=stream),
                          flush)
    vote_ms = sorted(vote_ms)[len(vote_ms) // 2]
    return depth_ms, mosaic_ms, model_points, vote_ms


def _single_e2e(st, torch, dev, stream, h, Lrgb, Rrgb, tL, tR, W, H, args, world, P):
    """End to end through the public API (see run_single)."""
    # end to end through the public API, run the way a video loop runs it:
    # every step uploads a pinned host RGB pair, matches it and reads the
    # refined map back; two device buffer sets let the upload of the next
    # pair (copy stream) and the read-back of the previous one (a second copy
    # stream) overlap the current match
    hL = torch.from_numpy(Lrgb).pin_memory()
    hR = torch.from_numpy(Rrgb).pin_memory()
    hout = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    dL = [torch.empty_like(tL) for _ in range(2)]
    dR = [torch.empty_like(tR) for _ in range(2)]
    dout = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in range(2)]
    dval = [torch.empty((H, W), dtype=torch.uint8, device=dev) for _ in range(2)]
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    for e in ev_done + ev_out:
        e.record(stream)

    def e2e_loop(n):
        for i in range(n):
            sl = i % 2
            up.wait_event(ev_done[sl])                 # match i-2 has read this input slot
            with torch.cuda.stream(up):
                dL[sl].copy_(hL, non_blocking=True)
                dR[sl].copy_(hR, non_blocking=True)
            ev_in[sl].record(up)
            stream.wait_event(ev_in[sl])
            stream.wait_event(ev_out[sl])               # read-back i-2 has left this output slot
            st.stereo_match(h, dL[sl], dR[sl], disp_final=dout[sl], valid=dval[sl], stream=stream)
            ev_done[sl].record(stream)
            down.wait_event(ev_done[sl])
            with torch.cuda.stream(down):
                hout[sl].copy_(dout[sl], non_blocking=True)
            ev_out[sl].record(down)
        for e in ev_out:
            stream.wait_event(e)

    e2e_loop(max(2, args.warmup))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    e2e_loop(args.steps)
    eb.record(stream)
    torch.cuda.synchronize()
    te = _max_over_ranks(torch, dev, ea.elapsed_time(eb) / 1e3, world)
    return world * args.steps * P / te / 1e9, te


def stage_bandwidth(stage_ms, W, H, D, wl):
    """Algorithmic bytes per stage of the single-pair path divided by the
    stage's event-timed milliseconds (GB/s).  Per pixel:
      statistics   reads 2 x 3 (RGB) or 2 x 1 (gray) B, writes both byte
                   images (2 B), left statistics (8 B), right statistics
                   (16 B) and clears both key maps (8 B);
      finalize     reads both key maps (8 B), writes the winner, LR and
                   sub-pixel maps (2 + 2 + 4 B) and reads the three parabola
                   costs (3 s B for a stored volume of s-byte elements);
      postprocess  3 rounds x (2 mask builds: read the 2 B map, write 4 x 4
                   bits; outlier test, radial and disc fill: read and write
                   the 2 B map): 3 x (2 x 4 + 3 x 4) = 60 B;
      refine       5 iterations x (Eq. 1-2: read packed o and d_prev, write
                   dt and b: 16 B; Eq. 3-4: read b, dt, counts, packed o,
                   write d_prev, packed o: 22 B) plus 11 candidates of s
                   bytes in each of the 4 o-updates (44 s B; none without a
                   volume) and the final map (4 B).
    The cost stage is the roofline line."""
    npix = W * H
    s = COST_BYTES[wl["cost"]]
    b = {"stats": npix * (6 + 2 + 8 + 16 + 8),
         "finalize": npix * (8 + 8 + 3 * s),
         "postprocess": npix * 60,
         "refine": npix * (5 * 38 + 44 * s + 4)}
    out = {}
    for k, nbytes in b.items():
        ms = stage_ms.get(k)
        if ms:
            out[k] = round(nbytes / (ms * 1e-3) / 1e9, 1)
    return out


def _depth_line(W, H, ms, peaks):
    """k_depth_points on the refined map: reads 4 B and writes 24 B (point and
    normal) per pixel; HBM-bound."""
    b = 28 * W * H
    gbs = b / (ms * 1e-3) / 1e9
    return {"kernel": "k_depth_points", "ms_median": round(ms, 4), "algorithmic_bytes": b,
            "achieved_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peaks["hbm_gbs"], 4),
            "note": "event-timed launch on the refined map, L2 flushed; not part of the step"}


# ------------------------------------------------------------- our arm: batch

def run_batched(args, wl, rank, world, dev, pairs):
    import torch
    import paper_2007_12623_b300 as st

    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    n = len(pairs)
    specs = [p[3] for p in pairs]
    maxW = max(s["W"] for s in specs)
    maxH = max(s["H"] for s in specs)
    maxD = max(s["D"] for s in specs)
    sp = st.stereo_default_params(max_width=maxW, max_height=maxH, num_disp=maxD,
                                  cost_dtype=COST_CODE[wl["cost"]], smooth_radius=wl["smooth_radius"])
    h = st.stereo_create(sp, max_batch=n)
    batch, host = [], []
    for (Lrgb, Rrgb, gt, s) in pairs:
        H, W = Lrgb.shape[:2]
        batch.append(dict(left=torch.from_numpy(Lrgb).to(dev), right=torch.from_numpy(Rrgb).to(dev),
                          d_min=0, num_disp=s["D"], win_radius=s["r"],
                          disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                          disp_sub=torch.empty((H, W), dtype=torch.float32, device=dev),
                          valid=torch.empty((H, W), dtype=torch.uint8, device=dev),
                          disp_final=torch.empty((H, W), dtype=torch.float32, device=dev)))
        host.append((torch.from_numpy(Lrgb).pin_memory(), torch.from_numpy(Rrgb).pin_memory(),
                     torch.empty((H, W), dtype=torch.float32).pin_memory()))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    tune = (st.stereo_autotune_batched(h, batch, stream=stream) if not args.no_autotune
            else dict(st.stereo_get_batch_config(h), note="default configuration, not tuned"))

    def step():
        st.stereo_match_batched(h, batch, use_graph=True, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        clk.wait_first_sample(step)
        torch.cuda.synchronize()
        launches0 = st.stereo_launch_count()
        step_ms = _timed_loop(torch, stream, args.steps, step, flush)
    launches = st.stereo_launch_count() - launches0
    t_max = _max_over_ranks(torch, dev, sum(step_ms) / 1e3, world)
    P = sum(s["W"] * s["H"] * s["D"] for s in specs)
    value = world * args.steps * P / t_max / 1e9
    stage_ms = _stage_pass(st, h, min(args.steps, 5), flush, step, st.STAGE_NAMES, stream)

    # end to end, as a stream of batches: the next batch's images go up from
    # pinned host memory (copy stream) into a staging set while the current
    # batch is matched, and the previous batch's refined maps come down from
    # a staging set (second copy stream); each step moves its inputs from
    # staging into the pairs' buffers and its outputs out of them with
    # device-to-device copies (the pairs' buffers, and so the batch's tables
    # and graph, stay the same)
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    stage_in = [[(torch.empty_like(b["left"]), torch.empty_like(b["right"])) for b in batch] for _ in range(2)]
    stage_out = [[torch.empty_like(b["disp_final"]) for b in batch] for _ in range(2)]
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    ev_down = [torch.cuda.Event() for _ in range(2)]
    for e in ev_used + ev_down:
        e.record(stream)

    def upload(sl):
        up.wait_event(ev_used[sl])                       # step sl - 2 has taken its inputs
        with torch.cuda.stream(up):
            for (sL, sR), (hL, hR, _) in zip(stage_in[sl], host):
                sL.copy_(hL, non_blocking=True)
                sR.copy_(hR, non_blocking=True)
        ev_up[sl].record(up)

    def e2e_batches(n):
        upload(0)
        for i in range(n):
            sl = i % 2
            if i + 1 < n:
                upload((i + 1) % 2)
            stream.wait_event(ev_up[sl])
            # device-to-device moves as elementwise kernels (x * 1, exact)
            # rather than DMA copies, which would queue behind the host
            # transfers on the copy engines (4 pairs: 1.135 -> 1.063 ms)
            for b, (sL, sR) in zip(batch, stage_in[sl]):
                torch.mul(sL, 1, out=b["left"])
                torch.mul(sR, 1, out=b["right"])
            ev_used[sl].record(stream)
            st.stereo_match_batched(h, batch, use_graph=True, stream=stream)
            stream.wait_event(ev_down[sl])               # read-back i - 2 has left this staging set
            for b, so in zip(batch, stage_out[sl]):
                torch.mul(b["disp_final"], 1, out=so)
            ev_out[sl].record(stream)
            down.wait_event(ev_out[sl])
            with torch.cuda.stream(down):
                for so, (_, _, ho) in zip(stage_out[sl], host):
                    ho.copy_(so, non_blocking=True)
            ev_down[sl].record(down)
        for e in ev_down:
            stream.wait_event(e)

    e2e_batches(max(2, args.warmup))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    e2e_batches(args.steps)
    eb.record(stream)
    torch.cuda.synchronize()
    te = _max_over_ranks(torch, dev, ea.elapsed_time(eb) / 1e3, world)
    e2e_value = world * args.steps * P / te / 1e9
    h.close()
    if rank != 0:
        return None
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = cost_kernel_roofline([(s["W"], s["H"], s["D"], s["r"], wl["cost"]) for s in specs],
                                stage_ms["cost_wta"], peaks, sm_count, "k_cost_batched",
                                KERNEL_TRAFFIC.get(args.workload))
    eq = 960 * 540 * 128 / P                      # one 960x540x128 pair's share of the work
    same = wl.get("same")
    line = _base_line(args, world, value, t_max, "f32", {
        "workload": args.workload, "pairs": n,
        "sizes": (f"{n} x {WORKLOADS[same]['W']}x{WORKLOADS[same]['H']} ({same} generator)" if same
                  else ("pairs %s of the 64-pair batch" % (wl["pick"],) if wl.get("pick")
                        else "16 each of 640x480, 960x540, 1280x720, 1920x1080")),
        "num_disp": sorted({s["D"] for s in specs}), "windows": sorted({2 * s["r"] + 1 for s in specs}),
        "cost_storage": wl["cost"], "smooth_radius": wl["smooth_radius"], "refine_iters": 5,
        "pix_disp_per_step": P, "parallelism": f"replicas x{world} (independent batches)",
        "l2": L2_NOTE + "; working set >> L2",
        "launch": "one stereo_match_batched per step, CUDA graph replay, persistent cost launch",
        "autotuned": tune})
    line.update({
        "ms_per_pair": round(t_max * 1e3 / args.steps / n, 4),
        "ms_per_960x540x128_equivalent": round(t_max * 1e3 / args.steps * eq, 4),
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "ms_per_step": round(te * 1e3 / args.steps, 4),
                "h2d_bytes_per_step": sum(2 * s["W"] * s["H"] * 3 for s in specs),
                "d2h_bytes_per_step": sum(s["W"] * s["H"] * 4 for s in specs),
                "mode": "stream of batches: upload of the next and read-back of the previous batch overlap the "
                        "current one (staging sets, device-to-device moves in the step); no L2 flush"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "paper_context": PAPER_CONTEXT,
    })
    return line


# ------------------------------------------------------------- our arm: soft

def _gray_f32(rgb):
    """ITU-R 601 luma in float (the soft-argmin form takes float images)."""
    return (rgb[..., 0] * 0.299 + rgb[..., 1] * 0.587 + rgb[..., 2] * 0.114).astype(np.float32)


def run_soft_step(args, wl, rank, world, dev):
    import torch
    import paper_2007_12623_b300 as st

    B, W, H, D, r, tau = wl["B"], wl["W"], wl["H"], wl["D"], wl["r"], wl["tau"]
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    data = [synth.tissue_pair(wl["seed"] + i, W, H, *wl["disp"]) for i in rank_pair_ids(wl, rank)]
    hL = torch.from_numpy(np.stack([_gray_f32(d[0]) for d in data])).pin_memory()
    hR = torch.from_numpy(np.stack([_gray_f32(d[1]) for d in data])).pin_memory()
    hG = torch.from_numpy(np.stack([d[2].astype(np.float32) for d in data])).pin_memory()
    tL, tR, tG = hL.to(dev), hR.to(dev), hG.to(dev)
    h = st.stereo_create(st.stereo_default_params(max_width=W, max_height=H, num_disp=D, soft_argmin=1))
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    hloss = torch.zeros(1, dtype=torch.float32).pin_memory()
    g = torch.empty((B, H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def train_step(L, R, G):
        L.requires_grad_(True)
        R.requires_grad_(True)
        L.grad = None
        R.grad = None
        ds = st.soft_argmin(L, R, h, 0, D, r, tau)
        st.stereo_l1_loss(h, ds.detach(), G, loss, g, stream=stream)
        ds.backward(g)
        return L.grad, R.grad

    def step():
        train_step(tL, tR, tG)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        clk.wait_first_sample(step, timeout=3.0)
        torch.cuda.synchronize()
        launches0 = st.stereo_launch_count()
        step_ms = _timed_loop(torch, stream, args.steps, step, flush)
    launches = st.stereo_launch_count() - launches0
    t_max = _max_over_ranks(torch, dev, sum(step_ms) / 1e3, world)
    P = B * W * H * D
    value = world * args.steps * P / t_max / 1e9

    # stage times of the backward of the last pair (separate pass)
    names = ("stats", "cost", "dA", "box_t1", "unused", "final")
    ds = st.soft_argmin(tL.detach(), tR.detach(), h, 0, D, r, tau)
    lse = torch.empty_like(ds)
    st.stereo_softargmin_fwd(h, tL.detach(), tR.detach(), 0, D, r, tau, ds, lse)
    gl, gr = torch.empty_like(ds), torch.empty_like(ds)
    bwd_ms = _stage_pass(st, h, min(args.steps, 5), flush,
                         lambda: st.stereo_softargmin_bwd(h, tL.detach(), tR.detach(), 0, D, r, tau, ds, lse,
                                                          g, gl, gr), names, stream)
    fwd_ms = _stage_pass(st, h, min(args.steps, 5), flush,
                         lambda: st.stereo_softargmin_fwd(h, tL.detach(), tR.detach(), 0, D, r, tau, ds, lse),
                         ("stats", "cost", "soft_fwd", "_a", "_b", "_c"), stream)

    # end to end, as a stream of training batches: the next batch's images
    # and ground truth go up from pinned host memory (copy stream) into the
    # other of two device sets while the current batch trains; every step
    # reads its loss back to pinned host memory
    up = torch.cuda.Stream(dev)
    sets = [(torch.empty_like(tL), torch.empty_like(tR), torch.empty_like(tG)) for _ in range(2)]
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]
    for e in ev_used:
        e.record(stream)

    def upload(sl):
        up.wait_event(ev_used[sl])                       # step sl - 2 is done with this set
        with torch.cuda.stream(up), torch.no_grad():
            for d_, h_ in zip(sets[sl], (hL, hR, hG)):
                d_.copy_(h_, non_blocking=True)
        ev_up[sl].record(up)

    def e2e_steps(n):
        upload(0)
        for i in range(n):
            sl = i % 2
            if i + 1 < n:
                upload((i + 1) % 2)
            stream.wait_event(ev_up[sl])
            L, R, G = sets[sl]
            train_step(L, R, G)
            hloss.copy_(loss, non_blocking=True)
            ev_used[sl].record(stream)

    e2e_steps(max(2, args.warmup))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    e2e_steps(args.steps)
    eb.record(stream)
    torch.cuda.synchronize()
    te = _max_over_ranks(torch, dev, ea.elapsed_time(eb) / 1e3, world)
    e2e_value = world * args.steps * P / te / 1e9
    h.close()
    if rank != 0:
        return None
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = soft_roofline(bwd_ms, W, H, D, peaks, sm_count, KERNEL_TRAFFIC.get(args.workload))
    line = _base_line(args, world, value, t_max, "f32", {
        "workload": args.workload, "batch": B, "width": W, "height": H, "num_disp": D,
        "window": 2 * r + 1, "tau": tau, "loss": "L1(d_soft, ground truth), mean over valid pixels",
        "step": "forward + loss + backward to both images (torch.autograd)",
        "parallelism": f"replicas x{world} (independent batches)",
        "l2": L2_NOTE + "; volumes >> L2"})
    line.update({
        "ms_per_pair": round(t_max * 1e3 / args.steps / B, 4),
        "stage_ms_last_pair": {"forward": {k: round(fwd_ms[k], 4) for k in ("stats", "cost", "soft_fwd")},
                               "backward": {k: round(v, 4) for k, v in bwd_ms.items() if k != "unused"}},
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "ms_per_step": round(te * 1e3 / args.steps, 4),
                "h2d_bytes_per_step": 3 * B * W * H * 4, "d2h_bytes_per_step": 4,
                "mode": "stream of batches: upload of the next batch overlaps the current training step "
                        "(two device sets); the loss is read back every step; no L2 flush"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "paper_context": PAPER_CONTEXT,
    })
    return line


# ------------------------------------------------------- CPU oracle leg

def _oracle_problem(wl):
    """(Lrgb, Rrgb, W, D, r, smooth radius) of the workload's first pair."""
    if wl["kind"] == "batched" and wl.get("same"):
        return _oracle_problem(WORKLOADS[wl["same"]])
    if wl["kind"] == "batched":
        L, R, gt, s = synth.batch_pair(16)               # a 960x540 pair of the batch
        return L, R, s["W"], s["D"], s["r"], wl["smooth_radius"]
    Lrgb, Rrgb, gt = make_pair(wl, 0)
    return Lrgb, Rrgb, wl["W"], wl["D"], wl["r"], wl.get("smooth_radius", 15)


def _oracle_params(wl, D, r, sr):
    import oracle
    return oracle.Params(d_min=wl.get("d_min", 0), num_disp=D, win_radius=r, smooth_radius=sr,
                         sampling=wl.get("sampling", 0))


def oracle_sample(wl, rows: int, problem=None):
    """Times the FP64 oracle on a bounded strip of the workload: `rows` output
    rows (plus window margins) across the full width.  Single-pair and batched
    workloads: the whole path; soft-argmin: forward + L1 loss + backward."""
    import oracle
    Lrgb, Rrgb, W, D, r, sr = problem or _oracle_problem(wl)
    H = Lrgb.shape[0]
    y0 = H // 2 - rows // 2 - r
    if wl["kind"] == "soft":
        Ls = _gray_f32(Lrgb)[y0:y0 + rows + 2 * r].astype(np.float64)
        Rs = _gray_f32(Rrgb)[y0:y0 + rows + 2 * r].astype(np.float64)
        gt = np.zeros_like(Ls)
        t0 = time.perf_counter()
        ds, lse, hv = oracle.softargmin_fwd(Ls, Rs, 0, D, r, wl["tau"])
        loss, g = oracle.l1_loss(ds, hv, gt)
        oracle.softargmin_bwd(Ls, Rs, 0, D, r, wl["tau"], g)
        dt = time.perf_counter() - t0
        return rows * W * D / dt / 1e9, dt, f"{W}x{rows} output rows (+{2 * r} margin rows), fwd+loss+bwd"
    Lg, Rg = oracle.gray(Lrgb), oracle.gray(Rrgb)
    Ls = np.ascontiguousarray(Lg[y0:y0 + rows + 2 * r])
    Rs = np.ascontiguousarray(Rg[y0:y0 + rows + 2 * r])
    p = _oracle_params(wl, D, r, sr)
    t0 = time.perf_counter()
    oracle.pipeline(Ls, Rs, p)
    dt = time.perf_counter() - t0
    return rows * W * D / dt / 1e9, dt, f"{W}x{rows} output rows (+{2 * r} margin rows) of a {W}-wide pair, D={D}"


def reference_config(name, wl, problem, rows):
    """The reference arm's own description: the same workload, evaluated by
    the single-threaded FP64 oracle on a strip of it."""
    Lrgb, Rrgb, W, D, r, sr = problem
    cfg = {"workload": name, "width": W, "height": Lrgb.shape[0], "num_disp": D, "d_min": wl.get("d_min", 0),
           "window": 2 * r + 1, "sampling": "chessboard" if wl.get("sampling", 0) else "full"}
    if wl["kind"] == "soft":
        cfg.update(tau=wl["tau"], step="soft-argmin forward + L1 loss + backward")
    else:
        cfg.update(smooth_radius=sr, refine_iters=5, step="whole path S0-S7")
    if wl["kind"] == "batched":
        cfg["pair"] = (f"a pair of the {wl['same']} workload (batched {wl['n']} at a time on the GPU)"
                       if wl.get("same") else "a 960x540 pair of the 64-pair batch")
    cfg.update(rows_per_step=rows, implementation="FP64 C oracle, single thread, host CPU",
               precision="f64")
    return cfg


def run_reference(args, wl):
    import oracle
    oracle.build()
    rows = args.oracle_rows
    problem = _oracle_problem(wl)
    W, D = problem[2], problem[3]
    for _ in range(args.warmup):
        oracle_sample(wl, max(2, rows // 4), problem)
    secs = []
    sample = ""
    for _ in range(args.steps):
        v, dt, sample = oracle_sample(wl, rows, problem)
        secs.append(dt)
    value = args.steps * rows * W * D / sum(secs) / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sum(secs) / args.steps * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA,
            "config": reference_config(args.workload, wl, problem, rows),
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: {sample}", **host_cpu()},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# Workloads measured beside the headline one in the default run (one GPU):
# name -> (steps, warmup).  Each runs exactly as its own --workload line
# would, with fewer steps.
SUB_WORKLOADS = {"perlin320": (200, 5), "tissue960_f16": (200, 5), "tissue960_none": (200, 5),
                 "tissue960_x4": (100, 5), "tissue960_x4_f16": (100, 5),
                 "tissue960_d192_f16": (200, 5), "tissue960_d192_bf16": (200, 5),
                 "tissue960_d192_f32": (200, 5), "paper960": (200, 5), "batch64": (6, 3), "soft8": (20, 3)}


def _sub_record(line):
    """The figures of a workload's line that the headline line carries."""
    keep = ("value", "unit", "ms_per_step", "ms_per_pair", "ms_per_960x540x128_equivalent", "dtype", "steps",
            "warmup", "gpu_launches", "stage_ms", "stage_ms_last_pair", "stage_gbs")
    rec = {k: line[k] for k in keep if k in line}
    rec["config"] = line["config"]
    r = line["roofline"]
    rec["roofline"] = {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel", "kernel_ms",
                                         "traffic") if k in r}
    rec["e2e"] = line["e2e"]
    rec["clocks"] = line["clocks"]
    return rec


def run_sub_workloads():
    """Every other workload, each in a process of its own (as a user would
    run it: `bench.py --workload NAME`), so that no state of the headline
    run (its cached device memory, the depth / mosaicking / voting extras)
    is left around it; the in-process runs measured 3-4 % slower than fresh
    processes on the same box."""
    out = {}
    for name, (steps, warmup) in SUB_WORKLOADS.items():
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", name, "--steps", str(steps),
               "--warmup", str(warmup), "--no-cpu-baseline", "--no-sub-workloads"]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode != 0 or not lines:
                out[name] = {"error": f"exit {r.returncode}: {r.stderr.strip()[-300:]}"}
                continue
            out[name] = _sub_record(json.loads(lines[-1]))
        except subprocess.TimeoutExpired:
            out[name] = {"error": "timed out"}
    return out


def host_cpu():
    """Host core count and CPU model (for the CPU baseline)."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="tissue960")
    ap.add_argument("--oracle-rows", type=int, default=8)
    ap.add_argument("--cpu-baseline-rows", type=int, default=96)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched workloads: the default unit configuration instead of the autotuner's")
    ap.add_argument("--no-sub-workloads", action="store_true",
                    help="default run only: skip the other workloads' records")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, wl)), flush=True)
        return

    subs = (world == 1 and args.workload == "tissue960" and not args.no_sub_workloads
            and "--workload" not in sys.argv)
    pairs = make_batch(rank_pair_ids(wl, rank), wl.get("same")) if wl["kind"] == "batched" else None
    import torch
    dev = torch.device(f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}")
    torch.cuda.set_device(dev)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    if wl["kind"] == "batched":
        line = run_batched(args, wl, rank, world, dev, pairs)
    elif wl["kind"] == "soft":
        line = run_soft_step(args, wl, rank, world, dev)
    else:
        line = run_single(args, wl, rank, world, dev)
    if subs:
        line["workloads"] = run_sub_workloads()
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            rows = args.cpu_baseline_rows if wl["kind"] != "soft" else max(4, args.cpu_baseline_rows // 8)
            v, dt, sample = oracle_sample(wl, rows)
            line["cpu_baseline"] = {"value": round(v, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": sample, "seconds": round(dt, 2), **host_cpu()}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
