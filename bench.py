#!/usr/bin/env python
"""Benchmark of the dense stereo-matching path (arXiv 2007.12623, Sec. II) on
B300.

One step = the whole path on one 960x540 RGB tissue pair (D = 128, 11x11
ZNCC window, FP32 cost volume, LR check, 3 outlier/hole-filling rounds,
5 refinement iterations with radius 15): gray -> window statistics ->
fused ZNCC + winner-take-all (left and right) + cost store -> sub-pixel / LR
-> outlier + hole filling -> improved Laplacian refinement.

Prints one JSON line (rank 0).  ``value`` is pixel-disparity evaluations per
second of the whole path (Gpix*disp/s) with inputs resident in device memory;
``e2e`` is the same metric through stereo_match with the RGB pair copied from
pinned host memory and the refined disparity copied back inside the timed
region.  ``--impl reference`` times the FP64 CPU oracle on a bounded sample
of the same workload instead.

Multi-GPU: one process per GPU (torchrun); every rank matches its own pair
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
    "tissue960": dict(W=960, H=540, D=128, r=5, cost="f32", smooth_radius=15, seed=synth.seed_for(1),
                      disp=(10.0, 110.0)),
    # 960x540, D = 0..191, 15x15 window, FP16 cost storage
    "tissue960_d192_f16": dict(W=960, H=540, D=192, r=7, cost="f16", smooth_radius=15,
                               seed=synth.seed_for(2), disp=(10.0, 170.0)),
    "tissue960_d192_bf16": dict(W=960, H=540, D=192, r=7, cost="bf16", smooth_radius=15,
                                seed=synth.seed_for(2), disp=(10.0, 170.0)),
    # 320x240 gray Perlin pair, D = 0..31, 5x5 smoothing
    "perlin320": dict(W=320, H=240, D=32, r=5, cost="f32", smooth_radius=2, seed=synth.seed_for(0),
                      disp=None),
}
COST_CODE = {"none": 0, "f32": 1, "f16": 2, "bf16": 3}
# DRAM bytes (read + write) of one k_cost_wta launch from an ncu capture of the
# current kernel on the same workload (profiles/k_cost_wta_<workload>.md);
# None where no capture of the current kernel exists.
COST_KERNEL_TRAFFIC = {"tissue960": 226.3e6}
COST_BYTES = {"none": 0, "f32": 4, "f16": 2, "bf16": 2}
METRIC = "Gpix*disp/s and ms per 960x540 pair (1 B300), % of roofline, vs oracle"
UNIT = "Gpix*disp/s"
L2_BYTES = 126 * 2 ** 20


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), sm_max_mhz=float(p.get("sm_max_mhz", 2032.0)),
                    source="measured")
    except Exception:
        return dict(hbm_gbs=6400.0, sm_max_mhz=2032.0, source="fallback")


def make_pair(wl, pair_index=0):
    if wl["disp"] is None:
        L, R, gt = synth.perlin_pair(wl["seed"] + pair_index, wl["W"], wl["H"])
        return np.stack([L] * 3, -1), np.stack([R] * 3, -1), gt
    return synth.tissue_pair(wl["seed"] + pair_index, wl["W"], wl["H"], *wl["disp"])


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
            for _ in range(20):
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

def cost_kernel_roofline(wl, cost_ms, peaks, sm_count, sm_mhz, traffic=None):
    """Roofline of the fused cost + winner-take-all kernel.

    Algorithmic work per pixel-disparity (p,d): 12 FP32/INT32 issue slots
    (1 product, 2 vertical + 2 horizontal sliding-sum updates, 2 for the
    numerator, 2 for rho, 2 for the winner compare/select, 1 for the store
    conversion) and s bytes of cost store (s = 4 FP32, 2 FP16/BF16).  Per
    pixel it also reads both gray images (2 B), both statistics maps (16 B) and
    writes both key maps (8 B).  The bound is whichever of the ALU time (12 ops
    on 128 lanes per SM per clock) and the HBM time is longer.
    """
    W, H, D = wl["W"], wl["H"], wl["D"]
    r = wl["r"]
    npix = (W - 2 * r) * (H - 2 * r)
    P = npix * D
    bytes_ = P * COST_BYTES[wl["cost"]] + W * H * (2 + 16 + 8)
    ops = 12 * P
    t_hbm = bytes_ / (peaks["hbm_gbs"] * 1e9)
    alu_peak = sm_count * 128 * peaks["sm_max_mhz"] * 1e6          # ops/s at max clock
    t_alu = ops / alu_peak
    dur = cost_ms * 1e-3
    if t_hbm >= t_alu:
        achieved = bytes_ / dur / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "kernel": "k_cost_wta", "algorithmic_bytes": bytes_,
                "peak_source": peaks["source"] + " (hbm_gbs)"}
    achieved = ops / dur / 1e12
    return {"bound": "alu", "achieved": round(achieved, 2), "peak": round(alu_peak / 1e12, 2),
            "unit": "Tops/s", "frac": round(achieved / (alu_peak / 1e12), 4), "traffic": traffic,
            "kernel": "k_cost_wta", "algorithmic_ops": ops,
            "peak_source": f"{sm_count} SMs x 128 lanes x {peaks['sm_max_mhz']:.0f} MHz"}


# ------------------------------------------------------------- our arm

def run_ours(args, wl, rank, world):
    import torch
    import paper_2007_12623_b300 as st

    dev = torch.device(f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}")
    torch.cuda.set_device(dev)
    W, H, D = wl["W"], wl["H"], wl["D"]
    Lrgb, Rrgb, gt = make_pair(wl, rank)
    tL = torch.from_numpy(Lrgb).to(dev)
    tR = torch.from_numpy(Rrgb).to(dev)
    sp = st.stereo_default_params(max_width=W, max_height=H, num_disp=D, win_radius=wl["r"],
                                  cost_dtype=COST_CODE[wl["cost"]], smooth_radius=wl["smooth_radius"])
    h = st.stereo_create(sp)
    outs = dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                disp_sub=torch.empty((H, W), dtype=torch.float32, device=dev),
                valid=torch.empty((H, W), dtype=torch.uint8, device=dev),
                disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        st.stereo_match(h, tL, tR, **outs, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = st.stereo_launch_count()
    with ClockSampler(dev.index) as clk:
        clk.wait_first_sample(lambda: step())   # keep the GPU busy until sampling starts
        launches0 = st.stereo_launch_count()
        for i in range(args.steps):
            flush.fill_(float(i))            # evict L2 between timed steps (not timed)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = st.stereo_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(step_ms) / 1e3
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    t_max = float(t.item())
    P = W * H * D
    value = world * args.steps * P / t_max / 1e9

    # per-stage times (separate, untimed-for-value runs with events between stages)
    st.stereo_set_stage_timing(h, True)
    nst = min(args.steps, 20)
    stage_sum = {n: 0.0 for n in st.STAGE_NAMES}
    for i in range(nst):
        flush.fill_(float(i))
        step()
        for k, v in st.stereo_get_stage_times(h).items():
            stage_sum[k] += v
    st.stereo_set_stage_timing(h, False)
    stage_ms = {k: v / nst for k, v in stage_sum.items()}

    # end to end through the public API: pinned host RGB in, refined map out
    hL = torch.from_numpy(Lrgb).pin_memory()
    hR = torch.from_numpy(Rrgb).pin_memory()
    hout = torch.empty((H, W), dtype=torch.float32).pin_memory()
    dL = torch.empty_like(tL)
    dR = torch.empty_like(tR)

    def e2e_step():
        dL.copy_(hL, non_blocking=True)
        dR.copy_(hR, non_blocking=True)
        st.stereo_match(h, dL, dR, disp_final=outs["disp_final"], valid=outs["valid"], stream=stream)
        hout.copy_(outs["disp_final"], non_blocking=True)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    e_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e_ms.append(a.elapsed_time(b))
    te = torch.tensor([sum(e_ms) / 1e3], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
    e2e_value = world * args.steps * P / float(te.item()) / 1e9
    h.close()

    if rank != 0:
        return None
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = clk.summary()
    roof = cost_kernel_roofline(wl, stage_ms["cost_wta"], peaks, sm_count, clocks.get("sm_mhz"),
                                COST_KERNEL_TRAFFIC.get(args.workload))
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max * 1e3 / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded tissue-texture generator standing in for the paper's videos)",
        "config": {"workload": args.workload, "width": W, "height": H, "num_disp": D,
                   "window": 2 * wl["r"] + 1, "cost_storage": wl["cost"],
                   "smooth_radius": wl["smooth_radius"], "refine_iters": 5, "pairs_per_gpu": 1,
                   "parallelism": f"replicas x{world} (independent pairs)",
                   "l2": "flushed between timed steps (256 MB write, untimed)"},
        "ms_per_pair": round(t_max * 1e3 / args.steps, 4),
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT,
                "ms_per_pair": round(float(te.item()) * 1e3 / args.steps, 4),
                "h2d_bytes_per_step": 2 * W * H * 3, "d2h_bytes_per_step": W * H * 4},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "paper_context": {"ms_per_keyframe_whole_pipeline": 76.3, "stereo_stage_ms": 15.9,
                          "zncc_ms_960x540x100": 5.0,
                          "hardware": "NVIDIA Titan X + Xeon X5472 (paper, Table III)"},
    }
    return line


# ------------------------------------------------------- CPU oracle leg

def oracle_sample(wl, rows: int):
    """Times the FP64 oracle's whole path on a bounded strip of the workload:
    `rows` output rows (plus window margins) across the full width."""
    import oracle
    Lrgb, Rrgb, gt = make_pair(wl, 0)
    Lg, Rg = oracle.gray(Lrgb), oracle.gray(Rrgb)
    y0 = wl["H"] // 2 - rows // 2 - wl["r"]
    Ls = np.ascontiguousarray(Lg[y0:y0 + rows + 2 * wl["r"]])
    Rs = np.ascontiguousarray(Rg[y0:y0 + rows + 2 * wl["r"]])
    p = oracle.Params(d_min=0, num_disp=wl["D"], win_radius=wl["r"], smooth_radius=wl["smooth_radius"])
    t0 = time.perf_counter()
    oracle.pipeline(Ls, Rs, p)
    dt = time.perf_counter() - t0
    P = rows * wl["W"] * wl["D"]
    return P / dt / 1e9, dt, f"{wl['W']}x{rows} output rows (+{2 * wl['r']} margin rows) of the workload"


def run_reference(args, wl):
    import oracle
    oracle.build()
    rows = args.oracle_rows
    for _ in range(args.warmup):
        oracle_sample(wl, max(2, rows // 4))
    vals, secs = [], []
    for _ in range(args.steps):
        v, dt, sample = oracle_sample(wl, rows)
        vals.append(v)
        secs.append(dt)
    value = args.steps * rows * wl["W"] * wl["D"] / sum(secs) / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sum(secs) / args.steps * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded tissue-texture generator)",
            "config": {"workload": args.workload, "width": wl["W"], "height": wl["H"],
                       "num_disp": wl["D"], "window": 2 * wl["r"] + 1},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: {sample}"},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


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
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, wl)), flush=True)
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, wl, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            v, dt, sample = oracle_sample(wl, args.cpu_baseline_rows)
            line["cpu_baseline"] = {"value": round(v, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": sample, "seconds": round(dt, 2)}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
