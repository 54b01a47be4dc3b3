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
SMS, SM_MAX_MHZ = 152, 2070.0

METRIC = "Winograd layer effective TFLOP/s at stated FP64 error; c-sweep evals/s vs plain"
# The point sets of the layer stacks: the paper's proposed sets for 2D
# F(4x4,3x3) (n = 6, c = 1.622) and F(6x6,3x3) (n = 8, c = 2, d = 1.003)
# (Table 8), which the sweep reproduces within its noise, and for contrast
# the integer / simple-fraction sets of Barabasz et al. the same table
# compares them with (P4 + {1/2, -2} and P8).
POINTSETS = {}


def _pointsets():
    from paper_2201_10369_gb300 import inputs
    inf = math.inf
    return {4: {"c_form": inputs.PROPOSED_SETS[(2, 6)] + [inf],
                "integer": inputs.COMPARISON_SETS[(2, 6)] + [inf]},
            6: {"c_form": inputs.PROPOSED_SETS[(2, 8)] + [inf],
                "integer": inputs.COMPARISON_SETS[(2, 8)] + [inf]}}


POINTSETS.update(_pointsets())
PTS4, PTS6 = POINTSETS[4]["c_form"], POINTSETS[6]["c_form"]
# End-to-end pipeline of the F(4x4) stack: sub-batches per VGG16 stage and
# the order the stages enter the pipeline.  The copies (~170 GB/s each way)
# bound it, and copy-out can only start once the first sub-batch is in and
# computed: small first units start it early, large stages split finely keep
# it fed, and the small deep stages are not split (their calls would be
# dominated by fixed per-call work).  Measured on GB300 (TFLOP/s): 2
# sub-batches for every stage, stages in order: 84.9; (8, 4, 2, 1, 1) in
# order: 89.1; (16, 8, 4, 2, 1): 86.0; (8, 4, 2, 1, 1), stages 4 and 5
# first: 90.4 (kept); uniform 4 or 8 sub-batches were slower than 2.
E2E_CHUNKS = (8, 4, 2, 1, 1)
E2E_ORDER = (4, 3, 0, 1, 2)
# contraction dtypes of the layer stacks (FP32 SIMT, then the tcgen05 forms)
STACK_DTYPES = ("f32", "bf16", "fp16", "split_bf16x3", "split_bf16x6")


def _stack_key(m, dt):
    return "f%dx%d" % (m, m) + ("" if dt == "f32" else "_" + dt)


# the layer stacks of one step: key -> (m, points, contraction dtype); the
# timed stacks run the c-form points (the kernels' work does not depend on
# the point values), the FP64 errors are stated for both point families
STACKS = {_stack_key(m, dt): (m, POINTSETS[m]["c_form"], dt)
          for m in (4, 6) for dt in STACK_DTYPES}
# 16-bit operand parts of each tensor-core dtype
TC_PARTS = {"bf16": 1, "fp16": 1, "split_bf16x3": 2, "split_bf16x6": 3}
# surrogate training: sweep labels of random instances of the sweep's sizes
# plus 1D F(m,5), m = 2..6 (d chosen so every size has valid subsets)
R5_SIZES = [(1, 2, 5, 1.0), (1, 3, 5, 1.0), (1, 4, 5, 1.0), (1, 5, 5, 2.478), (1, 6, 5, 1.229)]
SURROGATE_SAMPLES = 2_000_000
SURROGATE_EPOCHS = 200


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def reduce_max(values, world):
    """Per-rank timings reduced to their maximum over ranks (the bench's
    clock for N > 1 GPUs); the identity for one rank."""
    if world <= 1:
        return list(values)
    import torch
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def rank_seed(rank, layer):
    """Input seed of (rank, layer): every rank draws its own batch (weak
    scaling: per-GPU work fixed as ranks are added)."""
    return 1000 * rank + layer


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
    gpu_id = str(local_rank)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass

    # measured arithmetic peaks of the FP32 and FP64 pipes: the denominators
    # of every ALU roofline below
    pipe = measure_pipe_peaks(wino, gpu_id)

    # inputs resident in HBM (seeded per rank), outputs preallocated
    X, Wt = [], []
    for li, (C, H) in enumerate(layers):
        x, w = inputs.vgg_layer_device(C, H, N=N, seed=rank_seed(rank, li), device=dev)
        X.append(x)
        Wt.append(w)
    Y = {k: [torch.empty((N, C, H, H), device=dev) for C, H in layers] for k in STACKS}
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    cg = inputs.c_grid()
    sizes, masks = inputs.SWEEP_SIZES, inputs.sweep_masks()

    def stack(key):
        m, pts, dt = STACKS[key]
        for li in range(len(layers)):
            wino.wino_conv2d(X[li], Wt[li], Y[key][li], pts, m, 3, 1, dt)

    def sweep():
        return wino.wino_error_sweep(cg, sizes, masks, inputs.SWEEP_TRIALS, seed=rank)

    # planned persistent sweep of the same grid (mode autotuned, graph captured once)
    plan = wino.SweepPlan(sizes, wino.grid_instances(sizes, masks, cg), inputs.SWEEP_TRIALS,
                          seed=rank)
    # surrogate: labels from the sweep itself, trained once (reported, untimed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, Xs, ys = wino.surrogate_training_set(sizes + R5_SIZES, masks, SURROGATE_SAMPLES,
                                            inputs.SWEEP_TRIALS, seed=100 + rank)
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    model = wino.Surrogate(seed=rank)
    model.set_output_bias(float(ys.mean()))
    t0 = time.perf_counter()
    model.train(Xs, ys, batch=4096, epochs=SURROGATE_EPOCHS, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    guided = wino.GuidedSearch(model, sizes, masks, cg, inputs.SWEEP_TRIALS, seed=rank)

    # FP64 error of every (m, point family, contraction dtype) on every VGG16
    # stage (stated beside the throughput; untimed)
    fp64 = layer_errors(wino, X, Wt, layers, N, dev)
    torch.cuda.synchronize()

    # warm-up (the first calls also run the layer and sweep autotuners)
    for _ in range(args.warmup):
        for key in STACKS:
            stack(key)
        ex = sweep()
        plan.run(stream)
        guided.run()
    torch.cuda.synchronize()
    ex = np.where(np.isinf(ex), np.nan, ex)
    ex_rows = np.any(np.isfinite(ex), axis=2)
    exb = np.where(ex_rows, np.nanmin(np.where(ex_rows[:, :, None], ex, 1.0), axis=2), np.nan)

    names = ("wino_gemm", "input_transform", "output_transform", "filter_transform",
             "fused_layer", "sweep_eval", "sweep_prepare", "tc_gemm", "tc_transform")
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STACKS) + 1)]
          for _ in range(args.steps)]
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    wall = {"sweep": 0.0, "plan": 0.0, "guided": 0.0, "step": 0.0}
    guided_res = []
    clocks = ClockSampler(gpu_id)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wino.wino_profile_enable(True)
    for k in names:
        wino.wino_profile_read(k)
    launches0 = wino.wino_kernel_launches()
    torch.cuda.nvtx.range_push("timed")
    for s in range(args.steps):
        # L2 flush between steps; the stacks follow it in stream order (no
        # host synchronisation in between, so the GPU does not idle while the
        # first layer call is enqueued), outside the stacks' events
        ts = time.perf_counter()
        flush.fill_(float(s))
        # the stacks as a caller runs them: no per-kernel events (their times
        # give value and the stack figures) ...
        wino.wino_profile_enable(False)
        ev[s][0].record(stream)
        for i, key in enumerate(STACKS):
            stack(key)
            ev[s][i + 1].record(stream)
        # ... then once more with CUDA events around every library kernel
        # (the per-kernel durations of the rooflines); the events add ~60 us
        # per stack, which this pass keeps out of the stack times
        wino.wino_profile_enable(True)
        for key in STACKS:
            stack(key)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sweep()
        t1 = time.perf_counter()
        pev[s][0].record(stream)
        plan.run(stream)
        pev[s][1].record(stream)
        t2 = time.perf_counter()
        guided_res.append(guided.run())
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        wall["sweep"] += t1 - t0
        wall["plan"] += t2 - t1
        wall["guided"] += t3 - t2
        wall["step"] += t3 - ts
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = wino.wino_kernel_launches() - launches0
    wino.wino_profile_enable(False)
    prof = {k: wino.wino_profile_read(k) for k in names}
    clk = clocks.stop()
    tk = {key: sum(ev[s][i].elapsed_time(ev[s][i + 1]) for s in range(args.steps)) / 1e3
          for i, key in enumerate(STACKS)}
    t_plan = sum(a.elapsed_time(b) for a, b in pev) / 1e3
    times = ([tk[k] for k in STACKS] + [wall[k] for k in ("sweep", "plan", "guided", "step")] +
             [t_plan])
    times = reduce_max(times, world)
    for i, k in enumerate(STACKS):
        tk[k] = times[i]
    wall = dict(zip(("sweep", "plan", "guided", "step"), times[len(STACKS):len(STACKS) + 4]))
    t_plan = times[-1]
    fl = direct_flops(layers, N)
    tflops = {k: world * fl * args.steps / tk[k] / 1e12 for k in STACKS}
    n_inst = 503808
    vsw = world * n_inst * args.steps / wall["sweep"]
    vplan = world * n_inst * args.steps / wall["plan"]
    g_last = guided_res[-1]
    rows = np.isfinite(exb)
    ratios = g_last["best_err"][rows] / exb[rows]
    ratio, ratio_med = float(np.nanmax(ratios)), float(np.nanmedian(ratios))
    # rank of the guided best among the exhaustive row's errors (0 = the minimum)
    exf = np.where(np.isfinite(ex), ex, np.inf)
    ranks = np.array([(exf[s_, q_] < g_last["best_err"][s_, q_]).sum()
                      for s_, q_ in zip(*np.nonzero(rows))])

    # e2e: the F(4x4) FP32 stack through the public API with host buffers,
    # pipelined as a caller of the API would: the stages enter in the order
    # E2E_ORDER, stage l's batch as E2E_CHUNKS[l] sub-batches (wino_conv2d on a
    # batch slice computes the same outputs); a sub-batch's input is copied in
    # on one stream, it runs on a second once that input has landed, and its
    # output is copied out on a third once computed, so the host transfers
    # (the bound: ~200 GB/s each way) overlap compute and each other from the
    # first sub-batch on.  Timed from the first copy-in to the last copy-out
    # of each step, the device idle in between steps.
    xh = [x.cpu().pin_memory() for x in X]
    yh = [torch.empty(y.shape, dtype=y.dtype).pin_memory() for y in Y["f4x4"]]
    h2d = sum(x.numel() * 4 for x in X)
    d2h = sum(y.numel() * 4 for y in Y["f4x4"])
    s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    nl = len(layers)
    order = [li for li in E2E_ORDER if li < nl] + [li for li in range(nl) if li not in E2E_ORDER]
    chunks = [E2E_CHUNKS[li] if li < len(E2E_CHUNKS) else 1 for li in range(nl)]
    units = [(li, c * N // chunks[li], (c + 1) * N // chunks[li])
             for li in order for c in range(chunks[li])]
    ev_in = [torch.cuda.Event() for _ in units]
    ev_c = [torch.cuda.Event() for _ in units]
    m4, p4, dt4 = STACKS["f4x4"]
    te2e = 0.0
    for s in range(args.steps + 2):  # the first two untimed (the sub-batch shape's tuning)
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t_a = torch.cuda.Event(enable_timing=True)
        t_b = torch.cuda.Event(enable_timing=True)
        t_a.record(s_in)
        for u, (li, n0, n1) in enumerate(units):
            with torch.cuda.stream(s_in):
                X[li][n0:n1].copy_(xh[li][n0:n1], non_blocking=True)
            ev_in[u].record(s_in)
            s_comp.wait_event(ev_in[u])
            wino.wino_conv2d(X[li][n0:n1], Wt[li], Y["f4x4"][li][n0:n1], p4, m4, 3, 1, dt4,
                             stream=s_comp)
            ev_c[u].record(s_comp)
            s_out.wait_event(ev_c[u])
            with torch.cuda.stream(s_out):
                yh[li][n0:n1].copy_(Y["f4x4"][li][n0:n1], non_blocking=True)
        t_b.record(s_out)
        torch.cuda.synchronize()
        if s > 1:
            te2e += t_a.elapsed_time(t_b) / 1e3
    ve2e = world * fl * args.steps / te2e / 1e12

    # rooflines: each main kernel's algorithmic work / its CUDA-event time
    ctx = RoofCtx(wino, layers, N, args.steps, peaks, peak_src, pipe)
    roofs = {}
    for k, (ms, n) in prof.items():
        if n:
            r = kernel_roofline(k, ms, n, ctx)
            if r:
                roofs[k] = r
    roofs["sweep_plan"] = plan_roofline(t_plan, args.steps, ctx)
    per_size = sweep_per_size(wino, inputs, ctx, rank)
    comparison = paper_comparison(wino, inputs, ex, cg, masks, sizes)
    patterns = subset_tables(wino, inputs)
    orders = order_sweeps(wino, inputs, cg, sizes, masks, rank, pipe)
    plan_info = plan.info()
    plan.close()
    guided.close()
    model.close()

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": tflops["f4x4"], "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall["step"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": "VGG16 3x3 layer stack (C=64..512, H=224..14), N=32/GPU, FP32 Winograd "
                        "F(4x4,3x3) [value]; per step also the F(6x6,3x3) FP32 stack, the "
                        "BF16, FP16, split-BF16x3 and split-BF16x6 tensor-core stacks of both "
                        "sizes, the full point sweep (503808 instances x 1000 trials) "
                        "per-size and as one persistent graph launch, and the "
                        "surrogate-guided search of the same grid",
            "points": {"f%dx%d" % (m, m): {k: [float(v) for v in p] for k, p in fam.items()}
                       for m, fam in POINTSETS.items()},
            "timed_points": "c_form (the paper's proposed sets, Table 8 n = 6 and n = 8)",
            "global_batch": N * world,
            "parallelism": "dp%d" % world if world > 1 else "single",
            "timing": "per step each stack runs twice: once as a caller runs it (CUDA "
                      "events around the stack: value and stacks) and once with CUDA events "
                      "around every library kernel (the rooflines' per-kernel durations)",
            "l2": "256 MB flush between steps (untimed); each layer input > L2 except the "
                  "28x28/14x14 stages"},
        "roofline": roofs["fused_layer"],
        "rooflines": roofs,
        "pipe_peaks": pipe,
        "fp64_error": fp64,
        "stacks": {k: {"value": tflops[k], "unit": "TFLOP/s",
                       "ms_per_step": 1e3 * tk[k] / args.steps} for k in STACKS},
        "sweep": {"value": vsw, "unit": "evals/s", "instances": n_inst, "trials": 1000,
                  "ms_per_step": 1e3 * wall["sweep"] / args.steps, "path": "per-size kernels",
                  "per_size": per_size},
        "sweep_plan": {"value": vplan, "unit": "evals/s",
                       "ms_per_step": 1e3 * wall["plan"] / args.steps,
                       "graph_ms_per_step": 1e3 * t_plan / args.steps,
                       "mode": {1: "persistent", 2: "persistent3", 3: "per_size"}.get(
                           plan_info["mode"], plan_info["mode"]),
                       "grid": plan_info["grid"], "work_items": plan_info["items"]},
        "guided": {"wall_ms_per_step": 1e3 * wall["guided"] / args.steps,
                   "plain_sweep_wall_ms_per_step": 1e3 * wall["sweep"] / args.steps,
                   "speedup_vs_plain": wall["sweep"] / wall["guided"],
                   "evaluated_instances": g_last["evaluated"], "fallback_rows": g_last["fallback_rows"],
                   "rows": g_last["rows"], "max_best_err_ratio_vs_exhaustive": ratio,
                   "median_best_err_ratio_vs_exhaustive": ratio_med,
                   "rows_above_1.01x_exhaustive": int((ratios > 1.01).sum()),
                   "best_rank_in_exhaustive_row": {"median": float(np.median(ranks)),
                                                    "p90": float(np.percentile(ranks, 90)),
                                                    "max": int(ranks.max()),
                                                    "of": int(cg.size)},
                   "phase_ms": g_last["phase_ms"],
                   "training": {"samples": int(ys.numel()), "label_s": t_label,
                                "train_s": t_train, "epochs": SURROGATE_EPOCHS, "batch": 4096}},
        "e2e": {"value": ve2e, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "how": "F(4x4) FP32 stack via wino_conv2d from pinned host buffers; the "
                       "stages split into sub-batches, per sub-batch copy-in, layer and "
                       "copy-out on three streams (event-ordered), so transfers overlap compute",
                "sub_batches_per_layer": list(E2E_CHUNKS[:len(layers)]),
                "stage_order": [li for li in E2E_ORDER if li < len(layers)]},
        "gpu_launches": int(launches),
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "clocks": clk,
        "paper_comparison": comparison,
        "subset_patterns": patterns,
        "sweep_orders": orders,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(layers)
    print(json.dumps(line), flush=True)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo) and core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                name = ln.split(":", 1)[1].strip()
                if ln.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    name = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"model": name or "unknown", "nproc": os.cpu_count()}


def cpu_baseline(layers):
    """The oracle timed on the host cores on bounded samples of the step's
    workloads: the F(4x4) layer stack on 4 of the 32 images (all cores), the
    sweep on every 4th c (all cores) and on every 64th c (one core)."""
    v, dt, nth = oracle_layer_sample(layers)
    sw_rate, sw_dt, sw_nth, sw_n = oracle_sweep_sample(stride=4)
    s1_rate, s1_dt, s1_nth, s1_n = oracle_sweep_sample(stride=64, n_threads=1)
    return {
        "value": v, "unit": "TFLOP/s", "cores": nth, "kind": "oracle", "cpu": cpu_model(),
        "sample": "VGG16 5-layer F(4x4,3x3) stack on %d of the 32 images, one (layer, "
                  "image) per thread, %.1f s" % (ORACLE_IMAGES, dt),
        "sweep": {"value": sw_rate, "unit": "evals/s", "cores": sw_nth,
                  "sample": "every 4th c of the 4096-value grid, all sizes and subsets, "
                            "1000 trials (%d instances, %.1f s)" % (sw_n, sw_dt)},
        "sweep_1core": {"value": s1_rate, "unit": "evals/s", "cores": s1_nth,
                        "sample": "every 64th c of the 4096-value grid, all sizes and subsets, "
                                  "1000 trials (%d instances, %.1f s)" % (s1_n, s1_dt)}}


# launches of the pipe probes (about 60-100 ms each on a GB300)
PIPE_ITERS = {"fp32": 1 << 20, "fp32x2": 1 << 19, "fp64": 1 << 14}


def measure_pipe_peaks(wino, gpu_id, reps=3):
    """Best of `reps` launches of the library's FMA-throughput probe per pipe
    (wino_pipe_peak), with the SM clock sampled meanwhile; the FP32 peak is
    the larger of the scalar and packed forms."""
    for kind, iters in PIPE_ITERS.items():
        wino.wino_pipe_peak(kind, max(1, iters // 64))  # warm-up
    clocks = ClockSampler(gpu_id)
    clocks.start()
    out = {}
    for kind, iters in PIPE_ITERS.items():
        runs = [wino.wino_pipe_peak(kind, iters) for _ in range(reps)]
        out[kind] = {"tflops": max(r[0] for r in runs), "ms": min(r[1] for r in runs),
                     "iters": iters}
    out["clocks"] = clocks.stop()
    out["fp32_peak_tflops"] = max(out["fp32"]["tflops"], out["fp32x2"]["tflops"])
    out["fp64_peak_tflops"] = out["fp64"]["tflops"]
    out["how"] = ("wino_pipe_peak: 4 x 152 CTAs of 256 threads, 16 independent register "
                  "FMA chains per thread, best of %d launches (CUDA events)" % reps)
    return out


def layer_errors(wino, X, Wt, layers, N, dev):
    """Relative L1 error (and max error / max |y|) against the FP64 direct
    correlation of every (m, point family, contraction dtype) per VGG16
    stage: {f4x4: {c_form: {f32: {...}}}}."""
    import torch
    out = {}
    for li, (C, H) in enumerate(layers):
        y64 = torch.empty((N, C, H, H), dtype=torch.float64, device=dev)
        wino.wino_direct_conv_f64(X[li], Wt[li], y64, 1)
        yt = torch.empty((N, C, H, H), device=dev)
        for m, fam in POINTSETS.items():
            for pname, pts in fam.items():
                for dt in STACK_DTYPES:
                    wino.wino_conv2d(X[li], Wt[li], yt, pts, m, 3, 1, dt)
                    se, sr, me, mr = wino.wino_error_stats(yt, y64)
                    d = out.setdefault("f%dx%d" % (m, m), {}).setdefault(pname, {}).setdefault(
                        dt, {"rel_l1_per_layer": [], "max_rel_inf": 0.0})
                    d["rel_l1_per_layer"].append(se / sr)
                    d["max_rel_inf"] = max(d["max_rel_inf"], me / mr)
        del y64, yt
    return out


def paper_comparison(wino, inputs, ex, cg, masks, sizes):
    """Tables 7-8 from this run (untimed): per size, the relative error of
    Barabasz's set, of the paper's proposed set and of the best set the
    exhaustive sweep found (same trials), and the improvements over
    Barabasz's set beside the paper's."""
    out = {}
    # the wide 2D sizes (Table 8, n = 9, 10) at the paper's d, swept here
    # (untimed) for the comparison
    wide = [(2, 7, 3, 2.485), (2, 8, 3, 2.099)]
    ex_wide = wino.wino_error_sweep(cg, wide, masks, inputs.SWEEP_TRIALS, seed=0)
    for s, (dim, m, r, d) in enumerate(list(sizes) + wide):
        n = m + 2
        key = (dim, n)
        if key not in inputs.COMPARISON_SETS:
            continue
        ex_s = ex[s] if s < len(sizes) else ex_wide[s - len(sizes)]
        inf = math.inf
        pair = [inputs.COMPARISON_SETS[key] + [inf], inputs.PROPOSED_SETS[key] + [inf]]
        pn, prop = wino.wino_pointset_error((dim, m, r), pair, inputs.SWEEP_TRIALS, seed=0)
        pn_h, prop_h = wino.wino_pointset_error((dim, m, r), pair, inputs.SWEEP_TRIALS, seed=0,
                                                order="huffman")
        e = np.where(np.isfinite(ex_s), ex_s, np.nan)
        q, k = np.unravel_index(np.nanargmin(e), e.shape)
        best = float(e[q, k])
        out["%dd_n%d" % (dim, n)] = {
            "barabasz": float(pn), "paper_set": float(prop), "sweep_best": best,
            "sweep_best_mask": "%#04x" % int(masks[q]), "sweep_best_c": float(cg[k]),
            "d": d, "improvement_pct_paper_set": 100.0 * (pn - prop) / pn,
            "improvement_pct_sweep_best": 100.0 * (pn - best) / pn,
            "improvement_pct_printed": inputs.PAPER_IMPROVEMENT_PCT[key],
            "huffman_order": {"barabasz": float(pn_h), "paper_set": float(prop_h),
                              "improvement_pct_paper_set": 100.0 * (pn_h - prop_h) / pn_h}}
    # two-parameter (c, d) search of the paper's subset for the sizes whose
    # proposed set has a d: 128 d x 1024 c, log-spaced in [1.001, 4] x [0.25, 4]
    dg, cgg = np.geomspace(1.001, 4.0, 128), np.geomspace(0.25, 4.0, 1024)
    for dim, n, mask in CD_SEARCH:
        row = out.get("%dd_n%d" % (dim, n))
        if row is None:
            continue
        err = wino.cd_sweep(dim, n - 2, cgg, dg, [mask], inputs.SWEEP_TRIALS)[:, 0, :]
        e = np.where(np.isfinite(err), err, np.nan)
        i, k = np.unravel_index(np.nanargmin(e), e.shape)
        row["cd_search"] = {"mask": "%#04x" % mask, "c": float(cgg[k]), "d": float(dg[i]),
                            "err": float(e[i, k]),
                            "improvement_pct": 100.0 * (row["barabasz"] - e[i, k]) / row["barabasz"]}
    return out


GOLDEN = os.path.join(ROOT, "tests", "golden")


def _golden(name):
    """Rows of a '|'-separated golden file of the paper's printed values."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([v.strip() for v in line.split("|")])
    return rows


def subset_tables(wino, inputs):
    """Sec. 6.2 from this run's GPU sweep (untimed), c > 1 of the 4096-value
    grid, 1000 trials: Tables 2-4 (per base and subset, the c of least error
    and that error, beside the printed c) and Tables 5-6 (per base, the
    measured pattern -- the subset of least error -- and its win fraction,
    beside the printed pattern), through wino_subset_pattern."""
    cg = inputs.c_grid()
    cache = {}

    def sweep(dim, m, d, masks):
        key = (dim, m, d)
        if key not in cache:
            ms = np.array(sorted({b | s_ for b in (0x00, 0x20, 0x40, 0x60, 0x80) for s_ in range(16)
                                  if bin(b | s_).count("1") == m}), dtype=np.uint8)
            cache[key] = (ms, wino.wino_error_sweep(cg, [(dim, m, 3, d)], ms,
                                                    inputs.SWEEP_TRIALS, seed=0)[0])
        return cache[key]

    t234 = {}
    for lab, dim, m, d, mask, c, paper, _pin, cite in _golden("paper_subsets.txt"):
        dim, m, d, mask = int(dim), int(m), float(d), int(mask, 16)
        ms, err = sweep(dim, m, d, None)
        cands = wino.wino_subset_pattern(err, ms, cg, (dim, m, 3, d), mask & 0xF0, 1.0, 20.0)
        row = [x for x in cands if x["mask"] == mask][0]
        t234[lab] = {"mask": "%#04x" % mask, "best_c": row["best_c"], "rel_err": row["best_err"],
                     "printed_c": float(c), "printed_abs_err": float(paper), "cite": cite}
    t56 = {}
    for lab, dim, m, d, base, pat, cite in _golden("paper_patterns.txt"):
        dim, m, d, base = int(dim), int(m), float(d), int(base, 16)
        ms, err = sweep(dim, m, d, None)
        cands = wino.wino_subset_pattern(err, ms, cg, (dim, m, 3, d), base, 1.0, 20.0)
        t56[lab] = {"measured": "%#04x" % (cands[0]["mask"] & 0x0F),
                    "win_frac": cands[0]["win_frac"], "best_c": cands[0]["best_c"],
                    "printed": pat, "cite": cite,
                    "candidates": {"%#04x" % (x["mask"] & 0x0F): x["best_err"] for x in cands}}
    return {"tables_2_4": t234, "tables_5_6": t56,
            "how": "GPU sweep of every base | subset mask, c > 1 of the 4096-value grid, 1000 "
                   "trials; wino_subset_pattern per base"}


def order_smem_ops(dim, m, r):
    """Shared-memory value accesses of one trial of one instance in the
    Huffman-order kernels, every matrix entry counted as non-zero: a dot
    product of n terms stores n products, merges n - 1 times (two loads, one
    store) and loads its root: 4 n - 2."""
    a = m + r - 1
    dot = lambda n: 4 * n - 2  # noqa: E731
    if dim == 1:
        return a * dot(r) + a * dot(a) + m * dot(a)
    return a * r * dot(r) + a * a * dot(r) + 2 * a * a * dot(a) + m * a * dot(a) + m * m * dot(a)


def order_fp64_ops(dim, m, r):
    """FP64 multiplies and adds of one trial in the FP64-transform kernels
    (2 n - 1 per dot product of n terms, every entry counted as non-zero)."""
    a = m + r - 1
    dot = lambda n: 2 * n - 1  # noqa: E731
    if dim == 1:
        return a * dot(r) + a * dot(a) + m * dot(a)
    return a * r * dot(r) + a * a * dot(r) + 2 * a * a * dot(a) + m * a * dot(a) + m * m * dot(a)


def order_sweeps(wino, inputs, cg, sizes, masks, rank, pipe):
    """The full sweep grid in the two Huffman orders (Sec. 5), untimed by the
    step: wall time, kernel time and each kernel's bound -- the shared-memory
    pipe (128 B per SM per clock) for the FP32 form, the FP64 issue rate for
    the FP64-transform form."""
    out = {}
    n_inst = 0
    work = {"huffman": 0.0, "huffman_mixed": 0.0}
    for size in sizes:
        k = len(wino.valid_masks(size, masks)) * cg.size * inputs.SWEEP_TRIALS
        n_inst += len(wino.valid_masks(size, masks)) * cg.size
        work["huffman"] += 4.0 * k * order_smem_ops(*size[:3])
        work["huffman_mixed"] += 1.0 * k * order_fp64_ops(*size[:3])
    import torch
    sm_mhz = pipe["clocks"].get("sm_mhz") or SM_MAX_MHZ
    smem_peak = SMS * 128 * sm_mhz * 1e6 / 1e9
    fp64_peak = pipe["fp64_peak_tflops"] * 1e3 / 2  # Gop/s of separate multiplies or adds
    for order in ("huffman", "huffman_mixed"):
        wino.wino_error_sweep(cg[:64], sizes, masks, 100, seed=rank, order=order)  # warm-up
        torch.cuda.synchronize()
        wino.wino_profile_enable(True)
        t0 = time.perf_counter()
        wino.wino_error_sweep(cg, sizes, masks, inputs.SWEEP_TRIALS, seed=rank, order=order)
        dt = time.perf_counter() - t0
        ms, n = wino.wino_profile_read("sweep_order")
        wino.wino_profile_enable(False)
        sec = ms / 1e3
        if order == "huffman":
            ach = work[order] / sec / 1e9
            roof = {"bound": "smem", "unit": "GB/s", "achieved": ach, "peak": smem_peak,
                    "frac": ach / smem_peak, "traffic": None,
                    "peak_source": "derived: 152 SMs x 128 B/clock x %.0f MHz (the SM clock "
                                   "sampled during the pipe probes)" % sm_mhz,
                    "work": "4 B x (4n - 2) value accesses per n-term dot product"}
        else:
            ach = work[order] / sec / 1e9
            roof = {"bound": "fp64", "unit": "Gop/s", "achieved": ach, "peak": fp64_peak,
                    "frac": ach / fp64_peak, "traffic": None,
                    "peak_source": "measured FP64 FMA pipe probe (wino_pipe_peak), halved "
                                   "for separate multiplies and adds (of measured)",
                    "work": "2n - 1 FP64 multiplies and adds per n-term dot product"}
        out[order] = {"value": n_inst / dt, "unit": "evals/s", "wall_ms": 1e3 * dt,
                      "kernel_ms": ms, "launches": n, "instances": n_inst,
                      "trials": inputs.SWEEP_TRIALS, "roofline": roof}
    return out


# sizes (dim, n) whose proposed set in Tables 7-8 uses the d-group, with its subset
CD_SEARCH = [(1, 9, 0x7F), (1, 10, 0xFF), (2, 7, 0x4F), (2, 8, 0x5F), (2, 9, 0x7F),
             (2, 10, 0xFF)]


def _tiles(m, H, N):
    th = (H + m - 1) // m
    return N * th * th


class RoofCtx:
    """What the roofline helpers need: the library (for the transform
    matrices' non-zeros), the step's layers, and the peaks (HBM from the
    driver's measurement, FP32 / FP64 from the pipe probes)."""

    def __init__(self, wino, layers, N, steps, peaks, peak_src, pipe):
        self.wino, self.layers, self.N, self.steps = wino, layers, N, steps
        self.pipe = pipe
        sm = pipe["clocks"].get("sm_mhz")
        clk = (" at median SM clock %.0f MHz" % sm) if sm else ""
        self.fp32 = {"bound": "alu", "unit": "TFLOP/s", "peak": pipe["fp32_peak_tflops"],
                     "peak_source": "measured: FP32 FMA pipe probe (wino_pipe_peak, best of "
                                    "fma.rn.f32 / fma.rn.f32x2)%s (of measured)" % clk}
        self.fp64 = {"bound": "alu", "unit": "TFLOP/s", "peak": pipe["fp64_peak_tflops"],
                     "peak_source": "measured: FP64 FMA pipe probe (wino_pipe_peak, "
                                    "fma.rn.f64)%s (of measured)" % clk}
        self.hbm = {"bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"],
                    "peak_source": "copy bandwidth (of %s)" % peak_src}

    def nnz_at(self, m):
        """Non-zero entries of the FP32 A^T of the timed F(m x m, 3 x 3) points."""
        AT, _, _ = self.wino.wino_make_matrices(POINTSETS[m]["c_form"], m, 3)
        return int(np.count_nonzero(AT.astype(np.float32)))

    def stacks(self, kind):
        """(m, dtype) of the timed stacks that run `kind` ('f32' or 'tc')."""
        return [(m, dt) for m, _, dt in STACKS.values() if (dt == "f32") == (kind == "f32")]


def fp32_layer_work(ctx, m, C, H):
    """GEMM + output-transform flops of one FP32 layer launch (K = C):
    2 alpha^2 T C K for the contraction, 2 nnz(A^T) (alpha + m) per
    (tile, output channel) for A^T M A."""
    a = m + 2
    T = _tiles(m, H, ctx.N)
    return 2.0 * a * a * T * C * C + 2.0 * ctx.nnz_at(m) * (a + m) * T * C


def fp32_layer_bytes(ctx, m, C, H):
    """U read (alpha^2 T C floats), V read (alpha^2 C K), y written."""
    a = m + 2
    T = _tiles(m, H, ctx.N)
    return 4.0 * (a * a * T * C + a * a * C * C + ctx.N * C * H * H)


def tc_gemm_bytes(ctx, m, dt, C, H):
    """Every 16-bit part of U [F][Tp][Cp] and V [F][K][Cp] read once, M [F][K][T]
    written once in FP32 (K = C)."""
    F = (m + 2) ** 2
    T = _tiles(m, H, ctx.N)
    Tp = (T + 127) // 128 * 128
    Cp = (C + 63) // 64 * 64
    return F * (2.0 * TC_PARTS[dt] * (Tp * Cp + C * Cp) + 4.0 * T * C)


def tc_transform_bytes(ctx, m, dt, C, H):
    """The quantising transforms: x read, the 16-bit parts of U written; w
    read twice (maxima, then quantisation) and the parts of V written."""
    F = (m + 2) ** 2
    T = _tiles(m, H, ctx.N)
    Tp = (T + 127) // 128 * 128
    Cp = (C + 63) // 64 * 64
    p = TC_PARTS[dt]
    return 4.0 * ctx.N * C * H * H + 2.0 * p * F * Tp * Cp + 2 * 4.0 * 9 * C * C + 2.0 * p * F * C * Cp


def kernel_roofline(kernel, ms, n, ctx):
    """Algorithmic work of the step's launches of `kernel` / their summed
    CUDA-event time (= mean work per launch / mean launch time), against the
    kernel's bound."""
    per_step = n / ctx.steps
    sec = ms / 1e3 / ctx.steps  # event time per step
    L = ctx.layers
    work = None
    if kernel == "fused_layer":  # FP32 stacks: GEMM + fused output transform
        work, base = sum(fp32_layer_work(ctx, m, C, H) for m, _ in ctx.stacks("f32")
                         for C, H in L), ctx.fp32
    elif kernel == "input_transform":  # FP32 stacks: read x, write U
        work = sum(4.0 * (ctx.N * C * H * H + (m + 2) ** 2 * C * _tiles(m, H, ctx.N))
                   for m, _ in ctx.stacks("f32") for C, H in L)
        base = ctx.hbm
    elif kernel == "tc_gemm":
        # per frequency 2 T C K flops on 2 T C + 2 C K + 4 T K bytes: at most
        # 171 flop/byte (C = K = 512), below the ridge of the measured peaks
        # (~288), so every VGG stage is HBM-bound
        work = sum(tc_gemm_bytes(ctx, m, dt, C, H) for m, dt in ctx.stacks("tc") for C, H in L)
        base = ctx.hbm
    elif kernel == "tc_transform":
        work = sum(tc_transform_bytes(ctx, m, dt, C, H) for m, dt in ctx.stacks("tc")
                   for C, H in L)
        base = ctx.hbm
    elif kernel == "output_transform":  # tensor-core stacks: M read, y written
        work = sum(4.0 * ((m + 2) ** 2 * _tiles(m, H, ctx.N) * C + ctx.N * C * H * H)
                   for m, dt in ctx.stacks("tc") for C, H in L)
        base = ctx.hbm
    elif kernel == "sweep_eval":  # ONE full sweep per step, per-size kernels
        work, base = sweep_flops_total(), ctx.fp32
    if work is None:
        return None
    scale = 1e9 if base["unit"] == "GB/s" else 1e12
    ach = work / sec / scale
    return dict(kernel=kernel, bound=base["bound"], achieved=ach, peak=base["peak"],
                unit=base["unit"], frac=ach / base["peak"],
                traffic=kernel_traffic(kernel, ctx, per_step),
                peak_source=base["peak_source"], work_per_launch=work / per_step,
                launches_per_step=per_step, mean_launch_ms=ms / n)


def sweep_size_flops(dim, m, r, d, masks):
    """Dense FP32 flops of one size's full sweep (4096 c x 1000 trials)."""
    a = m + r - 1
    nmask = sum(1 for mk in masks if bin(int(mk)).count("1") == a - 2 and
                not (abs(d) == 1.0 and (int(mk) & 0x90)))
    if dim == 1:
        f = 2 * (a * r + a * a + m * a) + a
    else:
        f = 2 * (a * r * r + a * a * r) + 4 * a ** 3 + a * a + 2 * (m * a * a + m * m * a)
    return nmask * 4096 * 1000 * f


def sweep_per_size(wino, inputs, ctx, rank):
    """Each sweep size alone (untimed by the step): its k_sweep_eval time
    (CUDA events, the kernel only) and fraction of the FP32 peak."""
    cg, masks = inputs.c_grid(), inputs.sweep_masks()
    out = {}
    for size in inputs.SWEEP_SIZES:
        wino.wino_error_sweep(cg, [size], masks, inputs.SWEEP_TRIALS, seed=rank)  # warm-up
        wino.wino_profile_enable(True)
        wino.wino_profile_read("sweep_eval")
        wino.wino_error_sweep(cg, [size], masks, inputs.SWEEP_TRIALS, seed=rank)
        ms, n = wino.wino_profile_read("sweep_eval")
        wino.wino_profile_enable(False)
        fl = sweep_size_flops(*size, masks)
        ach = fl / (ms / 1e3) / 1e12
        out["%dd_F%d" % (size[0], size[1])] = {"kernel_ms": ms, "launches": n, "tflops": ach,
                                               "frac": ach / ctx.fp32["peak"]}
    return out


def plan_roofline(t_plan, steps, ctx):
    """The planned persistent sweep of the full grid (one graph replay per
    step, timed with CUDA events on its stream): one sweep's flops / time."""
    ach = sweep_flops_total() * steps / t_plan / 1e12
    return dict(kernel="sweep_plan (graph: k_sweep_prepare + k_sweep_persistent)",
                bound="alu", achieved=ach, peak=ctx.fp32["peak"], unit="TFLOP/s",
                frac=ach / ctx.fp32["peak"], traffic=None, peak_source=ctx.fp32["peak_source"],
                work_per_launch=sweep_flops_total(), launches_per_step=1.0,
                mean_launch_ms=1e3 * t_plan / steps)


# DRAM bytes (read + write) of one ncu capture of each kernel on a smaller
# case (profiles/), and the same case's algorithmic bytes; traffic of a bench
# launch = that ratio x the launch's algorithmic bytes (traffic grows in
# proportion to the bytes the launch must move).
NCU_TRAFFIC = {
    # k_gemm_otx_cl F(4x4) cluster tile shape split5, C = K = 512, 28x28,
    # N = 32: U read + V read + y written
    "fused_layer": (223.20e6, 36 * 1568 * 512 * 4 + 36 * 512 * 512 * 4
                    + 32 * 512 * 28 * 28 * 4),
    # k_tc_gemm split-BF16x6, C = K = 64, 224x224, N = 8: three 16-bit parts
    # of U and V read, M written (FP32)
    "tc_gemm": (535.54e6, 36 * (2 * 3 * (25216 * 64 + 64 * 64) + 4 * 25088 * 64)),
    # k_input_transform_blk F(4x4), C = 64, 224x224, N = 8: x read, U written
    "input_transform": (285.9e6, 334.0e6),
    # k_quant_input_mn split-BF16x6 F(4x4), C = 64, 224x224, N = 8: x read,
    # three 16-bit parts of U written (the filter kernels' bytes are small)
    "tc_transform": (390.28e6, 8 * 64 * 224 * 224 * 4 + 3 * 36 * 25088 * 64 * 2),
    # k_output_transform_r3 F(4x4), K = 64, 224x224, N = 8: M read, y written
    "output_transform": (300.7e6, 334.0e6),
}


def kernel_traffic(kernel, ctx, per_step):
    """Mean DRAM bytes per launch, scaled from the kernel's ncu capture, or
    None when no capture covers it."""
    if kernel not in NCU_TRAFFIC:
        return None
    meas, alg = NCU_TRAFFIC[kernel]
    L = ctx.layers
    if kernel == "fused_layer":
        b = sum(fp32_layer_bytes(ctx, m, C, H) for m, _ in ctx.stacks("f32") for C, H in L)
    elif kernel == "tc_gemm":
        b = sum(tc_gemm_bytes(ctx, m, dt, C, H) for m, dt in ctx.stacks("tc") for C, H in L)
    elif kernel == "input_transform":
        b = sum(4.0 * (ctx.N * C * H * H + (m + 2) ** 2 * C * _tiles(m, H, ctx.N))
                for m, _ in ctx.stacks("f32") for C, H in L)
    elif kernel == "tc_transform":
        b = sum(tc_transform_bytes(ctx, m, dt, C, H) for m, dt in ctx.stacks("tc") for C, H in L)
    else:  # output_transform
        b = sum(4.0 * ((m + 2) ** 2 * _tiles(m, H, ctx.N) * C + ctx.N * C * H * H)
                for m, dt in ctx.stacks("tc") for C, H in L)
    return meas / alg * b / per_step


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


def profile_case(name):
    """A small, bounded workload for ncu captures: inputs a few hundred MB
    (larger than L2), 4 runs of the case (1 warm-up + 3 to capture)."""
    import torch
    import paper_2201_10369_gb300 as wino
    from paper_2201_10369_gb300 import inputs
    wino.build()
    wino.load()
    base, shapes, nimg = name, [(64, 224)], 8
    if name.endswith("_vgg"):  # the five VGG16 stages, N=8
        base, shapes = name[:-4], inputs.VGG16_LAYERS
    elif name[-3:-1] == "_l":  # one VGG16 stage at the bench's N=32
        base, shapes, nimg = name[:-3], [inputs.VGG16_LAYERS[int(name[-1])]], 32
    if base in ("f4x4", "f6x6", "f4x4_bf16", "f4x4_split", "f4x4_x6", "f6x6_bf16", "f6x6_x6"):
        # one layer (64 ch, 224x224, N=8) unless a suffix says otherwise
        xs = [inputs.vgg_layer_device(C, H, N=nimg, seed=i) for i, (C, H) in enumerate(shapes)]
        ys = [torch.empty_like(x) for x, _ in xs]
        m, pts = (4, PTS4) if base.startswith("f4x4") else (6, PTS6)
        dt = {"bf16": "bf16", "split": "split_bf16x3",
              "x6": "split_bf16x6"}.get(base[5:], "f32")
        for _ in range(4):
            for (x, w), y in zip(xs, ys):
                wino.wino_conv2d(x, w, y, pts, m, 3, 1, dt)
    elif name == "sweep" or (name.startswith("sweep_") and name[6:7] in "12" and
                             name[7:8] == "d" and name[8:].isdigit()):
        # sweep: 2D F(4x4,3x3); sweep_<dim>d<m>: that size (the d of the sweep)
        dim, m = (2, 4) if name == "sweep" else (int(name[6]), int(name[8:]))
        size = [s_ for s_ in inputs.SWEEP_SIZES if s_[0] == dim and s_[1] == m][0]
        cg = inputs.c_grid()
        for _ in range(4):
            wino.wino_error_sweep(cg, [size], inputs.sweep_masks(), 1000, seed=0)
    elif name == "fp64_ref":
        # the FP64 direct reference and the FP64 error reduction on one VGG16
        # stage-2 shape (128 ch, 112x112, N = 2): 1.2 GFLOP in FP64
        x, w = inputs.vgg_layer_device(128, 112, N=2, seed=0)
        y = torch.empty_like(x)
        y64 = torch.empty(x.shape, dtype=torch.float64, device=x.device)
        wino.wino_conv2d(x, w, y, PTS4, 4, 3, 1, "f32")
        for _ in range(4):
            wino.wino_direct_conv_f64(x, w, y64, 1)
            wino.wino_error_stats(y, y64)
    elif name in ("sweep_huffman", "sweep_huffman_mixed"):
        cg = inputs.c_grid()
        for _ in range(4):
            wino.wino_error_sweep(cg, [(2, 4, 3, 1.0)], inputs.sweep_masks(), 1000, seed=0,
                                  order=name[6:])
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
                         "f4x4 | f6x6 | f4x4_bf16 | f4x4_split | f4x4_x6 | f6x6_bf16 | f6x6_x6 (VGG 64ch 224x224, N=8; "
                         "suffix _vgg: the five VGG16 stages, N=8; suffix _l0.._l4: that "
                         "VGG16 stage at N=32) | sweep (2D F(4x4), all masks, 4096 c) | "
                         "sweep_<dim>d<m> (that sweep size, e.g. sweep_1d4) | "
                         "sweep_huffman | sweep_huffman_mixed (the same in the Huffman "
                         "orders) | fp64_ref (FP64 direct reference and error reduction, "
                         "128 ch 112x112, N=2)")
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
