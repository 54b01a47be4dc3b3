#!/usr/bin/env python
"""Benchmark of the Winograd point-selection hot path on GB300.

One step = one pass of the hot path over one batch of synthetic input:
  (a) the VGG16-shaped 3x3 layer stack (C = 64/128/256/512/512 at
      H = 224/112/56/28/14, N = 32, stride 1, pad 1) with FP32 Winograd
      F(4x4,3x3) on the points {0, +-c, +-1/c, inf}, c = 1.622, and the same
      stack with F(6x6,3x3) on {0, +-c, +-1/c, -1/d, d, inf}, c = 2, d = 1.003;
  (b) the full point sweep: 1D F(m,3) m = 2..8 and 2D F(m x m,3x3) m = 2..6,
      every visited subset, 4096 log-spaced c in [0.05, 20], 1000 trials
      (503 808 instances).
value = effective TFLOP/s of the F(4x4) stack (direct-convolution FLOPs
2 N K C Ho Wo 9 divided by the measured time), with its FP64 error stated;
the F(6x6) stack and the sweep's evals/s are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs the same per-GPU workload (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0

C4, C6, D6 = 1.622, 2.0, 1.003
PTS4 = [0.0, -1 / C4, -C4, C4, 1 / C4, math.inf]
PTS6 = [0.0, -1 / C6, -C6, C6, 1 / C6, -D6, D6, math.inf]
METRIC = "Winograd layer effective TFLOP/s at stated FP64 error; c-sweep evals/s vs plain"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def direct_flops(layers, N):
    return sum(2.0 * N * C * C * H * H * 9 for C, H in layers)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [s.strip() for s in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------

ORACLE_IMAGES = 4  # images per layer in the oracle's bounded sample (of 32)


def oracle_layer_sample(layers, n_images=ORACLE_IMAGES):
    """Times the oracle's F(4x4) layers on `n_images` images per layer (a
    bounded sample of the N = 32 batch): one (layer, image) task per worker
    thread, all host cores.  Returns (effective TFLOP/s, seconds, threads)."""
    import concurrent.futures as cf
    import oracle
    from paper_2201_10369_gb300 import inputs
    oracle.build()
    tasks = []
    for C, H in layers:
        x, w = inputs.vgg_layer_host(C, H, N=n_images, seed=0)
        for n in range(n_images):
            tasks.append((np.ascontiguousarray(x[n:n + 1]), w))
    nth = min(len(tasks), os.cpu_count() or 1)

    def run(t):
        return oracle.wino_layer(t[0], t[1], 2, 1, PTS4, 4, 3)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(nth) as ex:
        list(ex.map(run, tasks))
    dt = time.perf_counter() - t0
    return direct_flops(layers, n_images) / dt / 1e12, dt, nth


def oracle_sweep_sample(stride=64, n_threads=None):
    """Times the oracle's sweep on every stride-th c of the full grid."""
    import oracle
    from paper_2201_10369_gb300 import inputs
    nth = n_threads or os.cpu_count() or 1
    cg = inputs.c_grid()
    t0 = time.perf_counter()
    e = oracle.error_sweep(cg, inputs.SWEEP_SIZES, inputs.sweep_masks(), inputs.SWEEP_TRIALS, 0,
                           c_stride=stride, n_threads=nth)
    dt = time.perf_counter() - t0
    n_inst = int(np.isfinite(e).sum() + np.isinf(e).sum())
    return n_inst / dt, dt, nth, n_inst


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2201_10369_gb300 import inputs
    layers = inputs.VGG16_LAYERS
    times, vals = [], []
    for i in range(args.warmup + args.steps):
        v, dt, nth = oracle_layer_sample(layers)
        if i >= args.warmup:
            times.append(dt)
            vals.append(v)
    value = direct_flops(layers, ORACLE_IMAGES) * len(times) / sum(times) / 1e12
    sw_rate, sw_dt, sw_nth, sw_n = oracle_sweep_sample(stride=16)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "VGG16 3x3 layer stack F(4x4,3x3), %d-image sample of the "
                               "N=32 batch (oracle, CPU)" % ORACLE_IMAGES,
                   "points": "c=1.622 {0,+-c,+-1/c,inf}"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": nth, "kind": "oracle",
                         "sample": "VGG16 5-layer F(4x4,3x3) stack on %d of the 32 images, one "
                                   "(layer, image) per thread" % ORACLE_IMAGES},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "sweep": {"value": sw_rate, "unit": "evals/s", "cores": sw_nth,
                  "sample": "every 16th c of the 4096-value grid, all sizes and subsets, "
                            "1000 trials (%d instances, %.1f s)" % (sw_n, sw_dt)},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2201_10369_gb300 as wino
    from paper_2201_10369_gb300 import inputs

    wino.build()
    wino.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if not wino.wino_device_ok():
        raise RuntimeError("libwino: no sm_103 device")
    peaks, peak_src = load_peaks()
    layers = inputs.VGG16_LAYERS
    N = inputs.VGG_BATCH
    stream = torch.cuda.current_stream()

    # inputs resident in HBM (seeded per rank), outputs preallocated
    X, Wt, Y4, Y6 = [], [], [], []
    for li, (C, H) in enumerate(layers):
        x, w = inputs.vgg_layer_device(C, H, N=N, seed=1000 * rank + li, device=dev)
        X.append(x)
        Wt.append(w)
        Y4.append(torch.empty((N, C, H, H), device=dev))
        Y6.append(torch.empty((N, C, H, H), device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    cg = inputs.c_grid()
    sizes, masks = inputs.SWEEP_SIZES, inputs.sweep_masks()

    def layers_f4():
        for li in range(len(layers)):
            wino.wino_conv2d(X[li], Wt[li], Y4[li], PTS4, 4, 3, 1)

    def layers_f6():
        for li in range(len(layers)):
            wino.wino_conv2d(X[li], Wt[li], Y6[li], PTS6, 6, 3, 1)

    def sweep():
        return wino.wino_error_sweep(cg, sizes, masks, inputs.SWEEP_TRIALS, seed=rank)

    # FP64 error of each layer (stated beside the throughput; untimed)
    layers_f4()
    layers_f6()
    torch.cuda.synchronize()
    fp64 = {"f4x4": [], "f6x6": []}
    for li in range(len(layers)):
        y64 = torch.empty(Y4[li].shape, dtype=torch.float64, device=dev)
        wino.wino_direct_conv_f64(X[li], Wt[li], y64, 1)
        for key, Y in (("f4x4", Y4), ("f6x6", Y6)):
            se, sr, me, mr = wino.wino_error_stats(Y[li], y64)
            fp64[key].append({"rel_l1": se / sr, "max_rel_inf": me / mr})
        del y64
    torch.cuda.synchronize()

    # warm-up
    for _ in range(args.warmup):
        layers_f4()
        layers_f6()
        sweep()
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    gpu_id = str(local_rank)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wino.wino_profile_enable(True)
    for k in ("wino_gemm", "input_transform", "output_transform", "filter_transform",
              "fused_layer", "sweep_eval", "sweep_prepare"):
        wino.wino_profile_read(k)
    launches0 = wino.wino_kernel_launches()
    for s in range(args.steps):
        flush.fill_(float(s))  # L2 flush between steps (outside the events)
        e0, e1, e2, e3 = ev[s]
        e0.record(stream)
        layers_f4()
        e1.record(stream)
        layers_f6()
        e2.record(stream)
        sweep()
        e3.record(stream)
    torch.cuda.synchronize()
    launches = wino.wino_kernel_launches() - launches0 - 0
    wino.wino_profile_enable(False)
    prof = {k: wino.wino_profile_read(k) for k in
            ("wino_gemm", "input_transform", "output_transform", "filter_transform",
             "fused_layer", "sweep_eval", "sweep_prepare")}
    clk = clocks.stop()
    t4 = sum(ev[s][0].elapsed_time(ev[s][1]) for s in range(args.steps)) / 1e3
    t6 = sum(ev[s][1].elapsed_time(ev[s][2]) for s in range(args.steps)) / 1e3
    tsw = sum(ev[s][2].elapsed_time(ev[s][3]) for s in range(args.steps)) / 1e3
    ttot = sum(ev[s][0].elapsed_time(ev[s][3]) for s in range(args.steps)) / 1e3
    if world > 1:
        t = torch.tensor([t4, t6, tsw, ttot], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t4, t6, tsw, ttot = t.tolist()
    fl = direct_flops(layers, N)
    v4 = world * fl * args.steps / t4 / 1e12
    v6 = world * fl * args.steps / t6 / 1e12
    n_inst = 503808
    vsw = world * n_inst * args.steps / tsw

    # e2e: the same F(4x4) stack through the public API with host buffers
    xh = [x.cpu().pin_memory() for x in X]
    yh = [torch.empty(y.shape, dtype=y.dtype).pin_memory() for y in Y4]
    h2d = sum(x.numel() * 4 for x in X)
    d2h = sum(y.numel() * 4 for y in Y4)
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for s in range(args.steps + 1):
        if s > 0:
            flush.fill_(float(s))
            ee[s - 1][0].record(stream)
        for li in range(len(layers)):
            X[li].copy_(xh[li], non_blocking=True)
            wino.wino_conv2d(X[li], Wt[li], Y4[li], PTS4, 4, 3, 1)
            yh[li].copy_(Y4[li], non_blocking=True)
        if s > 0:
            ee[s - 1][1].record(stream)
    torch.cuda.synchronize()
    te2e = sum(a.elapsed_time(b) for a, b in ee) / 1e3
    ve2e = world * fl * args.steps / te2e / 1e12

    # roofline of the dominant kernel of the F(4x4) + F(6x6) stacks
    layer_kernels = {k: v for k, v in prof.items() if k not in ("sweep_eval", "sweep_prepare")}
    dom = max(layer_kernels, key=lambda k: layer_kernels[k][0])
    dom_ms, dom_n = layer_kernels[dom]
    roof = roofline_for(dom, dom_ms, dom_n, layers, N, peaks, peak_src, clk)
    sw_ms, sw_n = prof["sweep_eval"]
    sweep_roof = sweep_roofline(sw_ms, sw_n, args.steps, clk)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": v4, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * ttot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": "VGG16 3x3 layer stack (C=64..512, H=224..14), N=32/GPU, FP32 "
                        "Winograd F(4x4,3x3); + F(6x6,3x3) stack + full point sweep per step",
            "points_f4x4": "{0,+-c,+-1/c,inf} c=1.622", "points_f6x6":
                "{0,+-c,+-1/c,-d,d,inf} c=2 d=1.003", "global_batch": N * world,
            "parallelism": "dp%d" % world if world > 1 else "single",
            "l2": "256 MB flush between steps (untimed); each layer input > L2 except "
                  "the 28x28/14x14 stages"},
        "fp64_error": {"f4x4_rel_l1_per_layer": [r["rel_l1"] for r in fp64["f4x4"]],
                       "f4x4_max_rel_inf": max(r["max_rel_inf"] for r in fp64["f4x4"]),
                       "f6x6_rel_l1_per_layer": [r["rel_l1"] for r in fp64["f6x6"]],
                       "f6x6_max_rel_inf": max(r["max_rel_inf"] for r in fp64["f6x6"])},
        "f6x6": {"value": v6, "unit": "TFLOP/s", "ms_per_step": 1e3 * t6 / args.steps},
        "f4x4_ms_per_step": 1e3 * t4 / args.steps,
        "sweep": {"value": vsw, "unit": "evals/s", "instances": n_inst, "trials": 1000,
                  "ms_per_step": 1e3 * tsw / args.steps, "roofline": sweep_roof},
        "roofline": roof,
        "e2e": {"value": ve2e, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        v, dt, nth = oracle_layer_sample(layers)
        sw_rate, sw_dt, sw_nth, sw_n = oracle_sweep_sample(stride=4)
        line["cpu_baseline"] = {
            "value": v, "unit": "TFLOP/s", "cores": nth, "kind": "oracle",
            "sample": "VGG16 5-layer F(4x4,3x3) stack on %d of the 32 images, one (layer, "
                      "image) per thread, %.1f s" % (ORACLE_IMAGES, dt),
            "sweep": {"value": sw_rate, "unit": "evals/s", "cores": sw_nth,
                      "sample": "every 4th c of the 4096-value grid, all sizes and subsets, "
                                "1000 trials (%d instances, %.1f s)" % (sw_n, sw_dt)}}
    print(json.dumps(line), flush=True)


def fp32_peak_tflops(clk):
    return SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12


def roofline_for(kernel, ms, n, layers, N, peaks, peak_src, clk):
    """Algorithmic work per launch of the dominant layer kernel / its mean
    event-timed duration."""
    if n == 0:
        return None
    # launches alternate F(4x4) and F(6x6) stacks: average the per-launch work
    works = []
    for m in (4, 6):
        a = m + 2
        for C, H in layers:
            th = (H + m - 1) // m
            T = N * th * th
            if kernel == "wino_gemm":
                works.append(2.0 * a * a * T * C * C)
            elif kernel == "input_transform":
                works.append(4.0 * (N * C * H * H + a * a * C * T))
            elif kernel == "output_transform":
                works.append(4.0 * (a * a * C * T + N * C * H * H))
            elif kernel == "fused_layer":
                works.append(2.0 * a * a * T * C * C)
            else:
                works.append(4.0 * (9 * C * C + a * a * C * C))
    per_launch = sum(works) / len(works)
    sec = ms / 1e3 / n
    if kernel in ("wino_gemm", "fused_layer"):
        peak = fp32_peak_tflops(clk)
        ach = per_launch / sec / 1e12
        return {"kernel": kernel, "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "work_per_launch": per_launch, "launches": n}
    peak = peaks["hbm_gbs"]
    ach = per_launch / sec / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "traffic": None, "peak_source": peak_src + " (of %s)" % peak_src,
            "work_per_launch": per_launch, "launches": n}


SWEEP_FLOPS_PER_TRIAL = None


def sweep_flops_total():
    """Dense FP32 flops of one full sweep: per trial and instance
    1D: 2(a r + a^2 + m a) + a; 2D: 2(a r^2 + a^2 r) + 4 a^3 + a^2 + 2(m a^2 + m^2 a)."""
    from paper_2201_10369_gb300 import inputs
    masks = inputs.sweep_masks()
    tot = 0.0
    for dim, m, r, d in inputs.SWEEP_SIZES:
        a = m + r - 1
        nmask = 0
        for mk in masks:
            pc = bin(int(mk)).count("1")
            if pc != a - 2 or (abs(d) == 1.0 and (int(mk) & 0x90)):
                continue
            nmask += 1
        if dim == 1:
            f = 2 * (a * r + a * a + m * a) + a
        else:
            f = 2 * (a * r * r + a * a * r) + 4 * a ** 3 + a * a + 2 * (m * a * a + m * m * a)
        tot += nmask * 4096 * 1000 * f
    return tot


def sweep_roofline(ms, n, steps, clk):
    if n == 0:
        return None
    sec = ms / 1e3 / steps  # the per-size eval launches of one sweep
    ach = sweep_flops_total() / sec / 1e12
    peak = fp32_peak_tflops(clk)
    return {"kernel": "sweep_eval", "bound": "alu", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
            "launches_per_sweep": n // steps}


def profile_case(name):
    """A small, bounded workload for ncu captures: inputs a few hundred MB
    (larger than L2), 4 runs of the case (1 warm-up + 3 to capture)."""
    import torch
    import paper_2201_10369_gb300 as wino
    from paper_2201_10369_gb300 import inputs
    wino.build()
    wino.load()
    if name in ("f4x4", "f6x6", "f4x4_bf16", "f4x4_split"):
        x, w = inputs.vgg_layer_device(64, 224, N=8, seed=0)
        y = torch.empty_like(x)
        m, pts = (4, PTS4) if name.startswith("f4x4") else (6, PTS6)
        dt = {"f4x4_bf16": "bf16", "f4x4_split": "split_bf16x3"}.get(name, "f32")
        for _ in range(4):
            wino.wino_conv2d(x, w, y, pts, m, 3, 1, dt)
    elif name == "sweep":
        cg = inputs.c_grid()
        for _ in range(4):
            wino.wino_error_sweep(cg, [(2, 4, 3, 1.0)], inputs.sweep_masks(), 1000, seed=0)
    else:
        raise SystemExit("unknown profile case " + name)
    torch.cuda.synchronize()
    print("profile case %s done" % name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    help="run one small workload a few times for an ncu capture: "
                         "f4x4 | f6x6 (VGG 64ch 224x224, N=8) | sweep (2D F(4x4), 15 masks)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
