#!/usr/bin/env python
"""Benchmark: linalg.matmul precision sweep at M = N = K = 8192 on GB300.

One step is one pass of the whole BF16 hot path over synthetic operands
already resident in HBM: operand prep (FP32 -> BF16 casts, B transposed to
K-major) and the tcgen05 GEMM with its epilogue, all through the C ABI.
`value` is the useful FLOP rate of the whole step (2*M*N*K / step time); the
roofline object times the GEMM kernel alone with CUDA events on its stream.
The FP32 operands (268 MB each) exceed the 129 MB L2, so no flush is needed.

Beside the headline the line carries: the rest of the precision sweep (FP8,
BF16x3, FP32 and the ratios to FP32), an end-to-end number through pinned
host buffers with the copies inside the timed region, the grouped-GEMM
config (one persistent launch replayed from a CUDA graph vs one launch per
GEMM), the convolution configs, the ResNet-style stack with schedules from
the learned cost model vs exhaustive search, and the FP64 oracle timed on
the host's cores on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nk|reference]

Under torchrun every rank runs its own independent problem (weak scaling);
rank 0 prints the line.  --impl reference times the FP64 CPU oracle alone.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 8192
METRIC = "TFLOP/s & % of tensor peak, matmul/conv2d, BF16/FP8 vs FP32 at stated error"
GEMM_SOURCES = ("paper_2307_16080_gb300/csrc/k_tc_gemm.cu", "paper_2307_16080_gb300/csrc/tc_ptx.cuh")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), float(p["hbm_gbs"]), "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


def source_sha():
    h = hashlib.sha256()
    for f in GEMM_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the kernel source as it is now (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[key]
        return rec["dram_bytes_per_launch"] if rec.get("source_sha256") == source_sha() else None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return len(os.sched_getaffinity(0))


def cpu_baseline(A, B, rows: int):
    """The FP64 oracle (as it stands) on `rows` output rows of the BF16 workload."""
    import oracle.nk_oracle as O
    t0 = time.perf_counter()
    O.matmul_precision(A[:rows], B, "bf16")
    dt = time.perf_counter() - t0
    flops = 2.0 * rows * B.shape[0] * B.shape[1]
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": host_threads(), "kind": "oracle",
            "sample": f"{rows} of {A.shape[0]} output rows of the BF16 {A.shape[0]}^3 matmul "
                      f"(bf16 rounding of both operands + FP64 numpy matmul), {dt:.1f} s"}


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle.nk_oracle as O
    from paper_2307_16080_gb300 import synth
    n = args.n
    A, B = synth.matmul_outlier(n, n, n)
    rows = args.ref_rows
    for _ in range(min(args.warmup, 1)):
        O.matmul_precision(A[:rows], B, "bf16")
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.matmul_precision(A[:rows], B, "bf16")
        times.append(time.perf_counter() - t0)
    flops = 2.0 * rows * n * n
    value = flops * len(times) / sum(times) / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"linalg.matmul precision sweep, BF16, M=N=K={n}; FP64 oracle on a sample"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": host_threads(), "kind": "oracle",
                             "sample": f"{rows} of {n} output rows per step"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_fn(torch, fn, reps, warm=2):
    st = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def graph_time(torch, fn, calls=10, reps=10):
    """Device time of one call: `calls` back-to-back calls captured into a
    CUDA graph, replayed `reps` times between CUDA events (no host work
    between the kernels, several calls per sample against the event clock's
    ~2 us granularity)."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(calls):
                fn()
    torch.cuda.current_stream().wait_stream(s)
    return time_fn(torch, g.replay, reps) / calls


def sweep_report(torch, nk, dev, a32, b32, c, flop, kern_tflops):
    """GEMM kernel throughput of the other precisions on the same operands."""
    out = {"bf16": kern_tflops}
    amax = torch.empty(2, device=dev)
    nk.nk_amax(a32, amax[0:1])
    nk.nk_amax(b32, amax[1:2])
    sc = torch.empty(2, device=dev)
    n = a32.shape[0]
    a8 = torch.empty(n, n, dtype=torch.uint8, device=dev)
    bt8 = torch.empty(n, n, dtype=torch.uint8, device=dev)
    nk.nk_cast_fp8(a32, amax[0:1], a8, scale_out=sc[0:1])
    nk.nk_cast_fp8(b32, amax[1:2], bt8, transpose=True, scale_out=sc[1:2])
    torch.cuda.synchronize()
    sa, sb = float(sc[0].item()), float(sc[1].item())
    ws8 = nk.workspace(nk.nk_matmul_workspace_size(a8, bt8.t(), c, "fp8"), dev)
    t8 = time_fn(torch, lambda: nk.nk_matmul(a8, bt8.t(), c, precision="fp8", scale_a=sa, scale_b=sb, ws=ws8), 10)
    out["fp8"] = flop / (t8 * 1e-3) / 1e12
    del a8, bt8, ws8
    wsx = nk.workspace(nk.nk_matmul_workspace_size(a32, b32, c, "bf16x3"), dev)
    tx = time_fn(torch, lambda: nk.nk_matmul(a32, b32, c, precision="bf16x3", ws=wsx), 5)
    out["bf16x3_with_prep"] = flop / (tx * 1e-3) / 1e12
    del wsx
    wsf = nk.workspace(nk.nk_matmul_workspace_size(a32, b32, c, "f32"), dev)
    tf = time_fn(torch, lambda: nk.nk_matmul(a32, b32, c, precision="f32", ws=wsf), 2, warm=1)
    out["f32"] = flop / (tf * 1e-3) / 1e12
    out["bf16_over_f32"] = out["bf16"] / out["f32"]
    out["fp8_over_f32"] = out["fp8"] / out["f32"]
    out["unit"] = "TFLOP/s (GEMM kernel; bf16x3 includes its split pass)"
    nk.nk_sync_status()
    return out


def e2e_report(torch, nk, dev, A, B, reps, nbuf=2):
    """Pinned host FP32 A, B in and host FP32 C out every step through the
    public API, with uploads, compute and downloads of consecutive steps on
    three streams (`nbuf` device buffer sets), as a user would pipeline them.
    The host link bounds it: on the GB300 machine pinned H2D copies reach about
    209 GB/s and D2H 192 GB/s whatever the number of streams or chunks, and
    329 GB/s together, so a step's 805 MB takes 2.45 ms at least; three or
    four buffer sets measure the same as two."""
    n = A.shape[0]
    a_h = torch.from_numpy(A).pin_memory()
    b_h = torch.from_numpy(B).pin_memory()
    c_h = [torch.empty(n, n).pin_memory() for _ in range(nbuf)]
    a32 = [torch.empty(n, n, device=dev) for _ in range(nbuf)]
    b32 = [torch.empty(n, n, device=dev) for _ in range(nbuf)]
    cc = [torch.empty(n, n, device=dev) for _ in range(nbuf)]
    a16 = torch.empty(n, n, dtype=torch.bfloat16, device=dev)
    bt16 = torch.empty(n, n, dtype=torch.bfloat16, device=dev)
    ws = nk.workspace(nk.nk_matmul_workspace_size(a16, bt16.t(), cc[0], "bf16"), dev)
    s_up, s_dn = torch.cuda.Stream(), torch.cuda.Stream()
    s_c = torch.cuda.current_stream()
    comp_done = [torch.cuda.Event() for _ in range(nbuf)]
    down_done = [torch.cuda.Event() for _ in range(nbuf)]
    up_done = [torch.cuda.Event() for _ in range(nbuf)]
    for j in range(nbuf):
        comp_done[j].record(s_c)
        down_done[j].record(s_c)

    def run(k):
        for i in range(k):
            j = i % nbuf
            with torch.cuda.stream(s_up):
                s_up.wait_event(comp_done[j])
                a32[j].copy_(a_h, non_blocking=True)
                b32[j].copy_(b_h, non_blocking=True)
                up_done[j].record(s_up)
            s_c.wait_event(up_done[j])
            s_c.wait_event(down_done[j])
            nk.nk_cast_bf16(a32[j], a16)
            nk.nk_cast_bf16(b32[j], bt16, transpose=True)
            nk.nk_matmul(a16, bt16.t(), cc[j], precision="bf16", ws=ws)
            comp_done[j].record(s_c)
            with torch.cuda.stream(s_dn):
                s_dn.wait_event(comp_done[j])
                c_h[j].copy_(cc[j], non_blocking=True)
                down_done[j].record(s_dn)
        torch.cuda.synchronize()

    run(2)
    t0 = time.perf_counter()
    run(reps)
    ms = (time.perf_counter() - t0) * 1e3 / reps
    nk.nk_sync_status()
    return {"value": 2.0 * n ** 3 / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "h2d_bytes_per_step": 2 * n * n * 4, "d2h_bytes_per_step": n * n * 4,
            "how": f"host wall clock over pipelined steps (upload / compute / download streams, {nbuf} buffer sets)"}


def grouped_report(torch, nk, synth, dev):
    """512 uneven BF16 GEMMs: one persistent launch replayed from a CUDA graph
    vs one nk_matmul launch per GEMM."""
    shapes = [tuple(int(v) for v in s) for s in synth.grouped_problems(512)]
    a = [torch.empty(M, K, device=dev).uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in shapes]
    bt = [torch.empty(N, K, device=dev).uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in shapes]
    c = [torch.empty(M, N, device=dev) for (M, N, K) in shapes]
    flop = float(sum(2.0 * M * N * K for (M, N, K) in shapes))
    groups, G = nk.make_groups(a, bt, c)
    from paper_2307_16080_gb300 import nk_tune as nt
    tuned, trep = nt.nk_grouped_tune(groups, G, reps=3)   # the autotuner picks the grouped tile
    plan = nk.nk_grouped_plan_create(groups, G, schedule=tuned)
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        nk.nk_grouped_plan_run(plan)
        with torch.cuda.graph(graph, stream=s):
            nk.nk_grouped_plan_run(plan)
    torch.cuda.current_stream().wait_stream(s)
    t_graph = time_fn(torch, graph.replay, 20)
    wss = [nk.workspace(nk.nk_matmul_workspace_size(a[g], bt[g].t(), c[g], "bf16"), dev) for g in range(G)]

    def per_gemm():
        for g in range(G):
            nk.nk_matmul(a[g], bt[g].t(), c[g], precision="bf16", ws=wss[g])
    t_loop = time_fn(torch, per_gemm, 5)
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)
    return {"groups": G, "useful_flop": flop, "persistent_graph_ms": t_graph, "per_gemm_launches_ms": t_loop,
            "persistent_graph_tflops": flop / (t_graph * 1e-3) / 1e12,
            "per_gemm_tflops": flop / (t_loop * 1e-3) / 1e12, "speedup": t_loop / t_graph,
            "schedule": list(tuned), "tuned_ms": trep.best_ms, "untuned_default_ms": trep.default_ms,
            "schedules_timed": trep.timed,
            "launches": {"persistent": 1, "per_gemm": G}}


def layer_roofline(N, H, W, C, F, KH, KW, stride, pad, ms):
    """min(tensor peak, HBM x arithmetic intensity) for one BF16 conv layer:
    2 B per input element (BF16 NHWC), 4 B per output element (FP32), 2 B per
    packed weight; achieved = FLOP / measured time."""
    bf16_peak, hbm, src = peaks()
    oh = (H + 2 * pad - KH) // stride + 1
    ow = (W + 2 * pad - KW) // stride + 1
    flop = 2.0 * N * oh * ow * F * KH * KW * C
    nbytes = 2.0 * N * H * W * C + 4.0 * N * oh * ow * F + 2.0 * KH * KW * C * F
    ai = flop / nbytes
    roof = min(bf16_peak, hbm * 1e-3 * ai)    # TFLOP/s
    achieved = flop / (ms * 1e-3) / 1e12
    return {"flop": flop, "bytes": nbytes, "ai_flop_per_byte": ai, "bound": "hbm" if roof < bf16_peak else "tensor",
            "roofline_tflops": roof, "achieved_tflops": achieved, "frac": achieved / roof,
            "peak_source": f"{src} (MEASURED_PEAKS.json)"}


def conv_batch32(torch, nk, synth, dev):
    """The same layer at batch 32 (the ResNet stack's first layers): FP32 on
    the CUDA cores vs BF16 on packed weights, graph-replayed device time."""
    I, W, bias = synth.conv_resnet_block(N=32)
    i32, w32, b32 = (torch.from_numpy(x).to(dev) for x in (I, W, bias))
    out = torch.empty(32, 56, 56, 64, device=dev)
    flop = 2.0 * 32 * 56 * 56 * 64 * 9 * 64
    g32 = graph_time(torch, lambda: nk.nk_conv2d_nhwc_hwcf(i32, w32, out, pad=(1, 1, 1, 1), bias=b32, relu=True),
                     calls=4, reps=5)
    i16, wp = i32.to(torch.bfloat16), nk.nk_conv2d_pack_weights(w32)
    ws = nk.workspace(nk.nk_conv2d_workspace_size(i16, wp, out, pad=(1, 1, 1, 1), precision="bf16"), dev)
    gp = graph_time(torch, lambda: nk.nk_conv2d_nhwc_hwcf(i16, wp, out, pad=(1, 1, 1, 1), precision="bf16",
                                                          bias=b32, relu=True, ws=ws))
    nk.nk_sync_status()
    return {"f32_ms": g32, "f32_tflops": flop / (g32 * 1e-3) / 1e12, "bf16_packed_ms": gp,
            "bf16_packed_tflops": flop / (gp * 1e-3) / 1e12, "bf16_packed_over_f32": g32 / gp}


def conv_report(torch, nk, synth, dev):
    """FP32 conv config (8x56x56x64, 3x3x64x64, s1 p1, bias + ReLU) on the
    CUDA cores, and the same layer in BF16 on the tensor cores."""
    I, W, bias = synth.conv_resnet_block()
    i32, w32, b32 = (torch.from_numpy(x).to(dev) for x in (I, W, bias))
    out = torch.empty(8, 56, 56, 64, device=dev)
    flop = 2.0 * 8 * 56 * 56 * 64 * 9 * 64
    t32 = time_fn(torch, lambda: nk.nk_conv2d_nhwc_hwcf(i32, w32, out, pad=(1, 1, 1, 1), bias=b32, relu=True), 20)
    i16 = i32.to(torch.bfloat16)
    ws = nk.workspace(nk.nk_conv2d_workspace_size(i16, w32, out, pad=(1, 1, 1, 1), precision="bf16"), dev)
    f16 = lambda: nk.nk_conv2d_nhwc_hwcf(i16, w32, out, pad=(1, 1, 1, 1), precision="bf16",  # noqa: E731
                                         bias=b32, relu=True, ws=ws)
    t16 = time_fn(torch, f16, 20)
    g32 = graph_time(torch, lambda: nk.nk_conv2d_nhwc_hwcf(i32, w32, out, pad=(1, 1, 1, 1), bias=b32, relu=True))
    g16 = graph_time(torch, f16)
    ws8 = nk.workspace(nk.nk_conv2d_workspace_size(i32, w32, out, pad=(1, 1, 1, 1), precision="fp8"), dev)
    g8 = graph_time(torch, lambda: nk.nk_conv2d_nhwc_hwcf(i32, w32, out, pad=(1, 1, 1, 1), precision="fp8",
                                                          bias=b32, relu=True, ws=ws8))
    wp = nk.nk_conv2d_pack_weights(w32)
    ws_p = nk.workspace(nk.nk_conv2d_workspace_size(i16, wp, out, pad=(1, 1, 1, 1), precision="bf16"), dev)
    gp = graph_time(torch, lambda: nk.nk_conv2d_nhwc_hwcf(i16, wp, out, pad=(1, 1, 1, 1), precision="bf16",
                                                          bias=b32, relu=True, ws=ws_p))
    nk.nk_sync_status()
    return {"f32_ms": t32, "f32_tflops": flop / (t32 * 1e-3) / 1e12, "bf16_ms": t16,
            "bf16_tflops": flop / (t16 * 1e-3) / 1e12, "bf16_over_f32": t32 / t16,
            "graph_f32_ms": g32, "graph_bf16_ms": g16, "graph_bf16_tflops": flop / (g16 * 1e-3) / 1e12,
            "graph_bf16_over_f32": g32 / g16,
            "graph_bf16_packed_ms": gp, "graph_bf16_packed_tflops": flop / (gp * 1e-3) / 1e12,
            "graph_bf16_packed_over_f32": g32 / gp,
            "roofline_bf16_packed": layer_roofline(8, 56, 56, 64, 64, 3, 3, 1, 1, gp),
            "graph_fp8_ms": g8, "graph_fp8_tflops": flop / (g8 * 1e-3) / 1e12, "graph_fp8_over_f32": g32 / g8,
            "batch32": conv_batch32(torch, nk, synth, dev),
            "note": "per call: host overhead included; graph: device time of calls replayed from a CUDA graph; "
                    "bf16 includes the per-call FP32 -> BF16 weight cast, bf16_packed takes weights packed once "
                    "by nk_conv2d_pack_weights, fp8 includes the per-call amax and E4M3 quantisation of I and W"}


def resnet_report(torch, synth, dev):
    """The 20-layer ResNet-style stack (BF16 conv, tensor cores) at batch 1,
    8, 32: total time with the built-in default schedules, with the cost
    model's top-5 (timed) pick, with the derivative-free (1+1) evolution
    strategy on the same budget of 5 timings, and with exhaustive search."""
    from paper_2307_16080_gb300 import costmodel
    from paper_2307_16080_gb300 import nk_tune as nt
    if not os.path.exists(costmodel.MODEL_PATH):
        return None
    params, _, _ = costmodel.load_model()
    P = torch.from_numpy(params).to(dev)
    out = {}
    for b in (1, 8, 32):
        tot = {"default_ms": 0.0, "model_top5_ms": 0.0, "evolution5_ms": 0.0, "exhaustive_ms": 0.0, "flop": 0.0}
        timed = {"model": 0, "evolution": 0, "exhaustive": 0}
        picks = []
        for L in synth.resnet_stack(b):
            p = nt.conv_problem(L["N"], L["H"], L["W"], L["C"], L["F"], L["KH"], L["KW"], L["stride"], L["pad"])
            _, ex = nt.nk_tune(p, nt.NK_TUNE_EXHAUSTIVE, reps=3)
            pick, mo = nt.nk_tune(p, nt.NK_TUNE_MODEL_TOPK, topk=5, params=P, reps=3)
            picks.append(pick)
            _, es = nt.nk_tune(p, nt.NK_TUNE_EVOLUTION, topk=5, reps=3)
            tot["default_ms"] += ex.default_ms
            tot["exhaustive_ms"] += ex.best_ms
            tot["model_top5_ms"] += mo.best_ms
            tot["evolution5_ms"] += es.best_ms
            timed["model"] += mo.timed
            timed["evolution"] += es.timed
            timed["exhaustive"] += ex.timed
            oh = (L["H"] + 2 * L["pad"] - L["KH"]) // L["stride"] + 1
            tot["flop"] += 2.0 * b * oh * oh * L["F"] * L["KH"] * L["KW"] * L["C"]
        tot["model_regret"] = tot["model_top5_ms"] / tot["exhaustive_ms"] - 1
        tot["default_regret"] = tot["default_ms"] / tot["exhaustive_ms"] - 1
        tot["evolution_regret"] = tot["evolution5_ms"] / tot["exhaustive_ms"] - 1
        tot["model_tflops"] = tot["flop"] / (tot["model_top5_ms"] * 1e-3) / 1e12
        tot["schedules_timed"] = timed
        tot["stack_graph"] = stack_graph(torch, synth, dev, b, picks, tot["flop"])
        out[f"batch{b}"] = tot
    nt.nk_tune_release()
    return out


def stack_graph(torch, synth, dev, batch, picks, flop):
    """The whole 20-layer stack through the public API, as a user deploys it:
    weights packed to BF16 once (nk_conv2d_pack_weights), then each layer an
    nk_conv2d_nhwc_hwcf call (BF16 input, bias + ReLU, the cost model's pick
    as schedule), all 20 captured into one CUDA graph and replayed."""
    import paper_2307_16080_gb300.nk as nk
    calls = []
    for li, (L, sched) in enumerate(zip(synth.resnet_stack(batch), picks)):
        oh = (L["H"] + 2 * L["pad"] - L["KH"]) // L["stride"] + 1
        i = torch.empty(L["N"], L["H"], L["W"], L["C"], device=dev).uniform_(0, 1).to(torch.bfloat16)
        w = nk.nk_conv2d_pack_weights(torch.empty(L["KH"], L["KW"], L["C"], L["F"], device=dev).normal_(
            0, (2.0 / (L["KH"] * L["KW"] * L["C"])) ** 0.5))
        bias = torch.empty(L["F"], device=dev).uniform_(-0.1, 0.1)
        o = torch.empty(L["N"], oh, oh, L["F"], device=dev)
        st, pad = (L["stride"],) * 2, (L["pad"],) * 4
        ws = nk.workspace(nk.nk_conv2d_workspace_size(i, w, o, st, (1, 1), pad, "bf16", sched), dev)
        calls.append((i, w, o, st, pad, bias, sched, ws))

    def forward():
        for (i, w, o, st, pad, bias, sched, ws) in calls:
            nk.nk_conv2d_nhwc_hwcf(i, w, o, st, (1, 1), pad, "bf16", bias=bias, relu=True, schedule=sched, ws=ws)
    ms = graph_time(torch, forward, calls=2, reps=10)
    nk.nk_set_pdl(False)   # the same graph captured with plain stream ordering between kernels
    ms_serial = graph_time(torch, forward, calls=2, reps=10)
    nk.nk_set_pdl(True)
    nk.nk_sync_status()
    kernels = sum(2 if sched[5] > 1 else 1 for sched in picks)   # split-K adds its reduce
    # the stack's roofline time: each layer at min(tensor peak, HBM x its arithmetic intensity)
    roof_ms = 0.0
    for L in synth.resnet_stack(batch):
        r = layer_roofline(L["N"], L["H"], L["W"], L["C"], L["F"], L["KH"], L["KW"], L["stride"], L["pad"], 1.0)
        roof_ms += r["flop"] / (r["roofline_tflops"] * 1e12) * 1e3
    return {"ms": ms, "tflops": flop / (ms * 1e-3) / 1e12, "kernels_per_forward": kernels,
            "ms_without_pdl": ms_serial, "pdl_speedup": ms_serial / ms,
            "roofline_ms": roof_ms, "frac_of_roofline": roof_ms / ms,
            "how": "20 nk_conv2d calls on packed BF16 weights (one conv kernel each) in one CUDA graph, device time; "
                   "ms with programmatic dependent launch (default), ms_without_pdl with nk_set_pdl(0)"}


def grouped_conv_report(torch, nk, synth, dev, batch=8):
    """The 20 ResNet-stack layer shapes at batch 8 as independent convolutions
    (each with its own input): one persistent launch of all 20 (a grouped
    conv plan) against 20 nk_conv2d calls with built-in schedules, both
    replayed from CUDA graphs."""
    convs, flop = [], 0.0
    for L in synth.resnet_stack(batch):
        oh = (L["H"] + 2 * L["pad"] - L["KH"]) // L["stride"] + 1
        i = torch.empty(L["N"], L["H"], L["W"], L["C"], device=dev).uniform_(0, 1).to(torch.bfloat16)
        w = nk.nk_conv2d_pack_weights(torch.empty(L["KH"], L["KW"], L["C"], L["F"], device=dev).normal_(0, 0.05))
        o = torch.empty(L["N"], oh, oh, L["F"], device=dev)
        convs.append(dict(I=i, W=w, O=o, stride=(L["stride"],) * 2, pad=(L["pad"],) * 4, relu=True,
                          bias=torch.zeros(L["F"], device=dev)))
        flop += 2.0 * L["N"] * oh * oh * L["F"] * L["KH"] * L["KW"] * L["C"]
    groups, G = nk.make_conv_groups(convs)
    from paper_2307_16080_gb300 import nk_tune as nt
    tuned, trep = nt.nk_conv2d_grouped_tune(groups, G, reps=3)   # the autotuner picks the tile
    plan = nk.nk_conv2d_grouped_plan_create(groups, G, schedule=tuned)
    t_grouped = graph_time(torch, lambda: nk.nk_grouped_plan_run(plan), calls=2, reps=10)
    nk.nk_grouped_plan_destroy(plan)
    wss = [nk.workspace(nk.nk_conv2d_workspace_size(d["I"], d["W"], d["O"], d["stride"], (1, 1), d["pad"], "bf16"),
                        dev) for d in convs]

    def separate():
        for d, ws in zip(convs, wss):
            nk.nk_conv2d_nhwc_hwcf(d["I"], d["W"], d["O"], d["stride"], (1, 1), d["pad"], "bf16", bias=d["bias"],
                                   relu=True, ws=ws)
    t_sep = graph_time(torch, separate, calls=2, reps=10)
    nk.nk_sync_status()
    return {"groups": G, "batch": batch, "flop": flop, "one_launch_ms": t_grouped,
            "one_launch_tflops": flop / (t_grouped * 1e-3) / 1e12, "separate_launches_ms": t_sep,
            "separate_tflops": flop / (t_sep * 1e-3) / 1e12, "speedup": t_sep / t_grouped,
            "schedule": list(tuned), "schedules_timed": trep.timed, "untuned_default_ms": trep.default_ms,
            "how": "device time of CUDA-graph replays; grouped: per-tap kernel, tile from nk_conv2d_grouped_tune"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nk", choices=["nk", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--ref-rows", type=int, default=16)
    ap.add_argument("--cpu-rows", type=int, default=64)
    ap.add_argument("--no-sweep", action="store_true", help="skip the FP8/BF16x3/FP32 sweep")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-check", action="store_true", help="skip the sampled accuracy check")
    ap.add_argument("--no-extra", action="store_true", help="skip the grouped / conv / ResNet reports")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    import paper_2307_16080_gb300.nk as nk
    from paper_2307_16080_gb300 import nk_tune as nt
    from paper_2307_16080_gb300 import shard, synth

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    n = args.n
    A, B = synth.matmul_outlier(n, n, n)            # one independent problem per rank (weak scaling)
    a32 = torch.from_numpy(A).to(dev)
    b32 = torch.from_numpy(B).to(dev)
    c = torch.empty(n, n, device=dev)
    a16 = torch.empty(n, n, dtype=torch.bfloat16, device=dev)
    bt16 = torch.empty(n, n, dtype=torch.bfloat16, device=dev)   # B^T, K-major
    st = torch.cuda.current_stream()
    ws = nk.workspace(nk.nk_matmul_workspace_size(a16, bt16.t(), c, "bf16"), dev)
    sched = nt.nk_default_schedule(nt.matmul_problem(n, n, n, "bf16"))

    def step(ev_k=None):
        nk.nk_cast_bf16(a32, a16)
        nk.nk_cast_bf16(b32, bt16, transpose=True)
        if ev_k:
            ev_k[0].record(st)
        nk.nk_matmul(a16, bt16.t(), c, precision="bf16", ws=ws)
        if ev_k:
            ev_k[1].record(st)

    for _ in range(args.warmup):
        step()
    nk.nk_sync_status()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(st)
    for i in range(args.steps):
        step(kev[i])
    e1.record(st)
    barrier()
    clk = clocks.stop()
    nk.nk_sync_status()
    ms = shard.max_over_ranks(e0.elapsed_time(e1))
    kern_ms = sum(a.elapsed_time(b) for a, b in kev) / args.steps
    flop = 2.0 * n * n * n
    value = flop * args.steps * world / (ms * 1e-3) / 1e12
    kern_tflops = flop / (kern_ms * 1e-3) / 1e12

    accuracy = {}
    if rank == 0 and not args.no_check:
        import oracle.nk_oracle as O
        rows = np.sort(synth.raw_u64(77, 1, 32) % np.uint64(n)).astype(np.int64)
        got = c[torch.from_numpy(rows).to(dev)].cpu().numpy()
        accuracy["err_vs_bf16_inputs_sampled"] = O.rel_frobenius(got, O.matmul(O.bf16_rn(A[rows]), O.bf16_rn(B)))
        accuracy["err_vs_fp32_inputs_sampled"] = O.rel_frobenius(got, O.matmul(A[rows], B))
        accuracy["rows"] = len(rows)

    sweep = None if args.no_sweep else sweep_report(torch, nk, dev, a32, b32, c, flop, kern_tflops)
    e2e = None
    if not args.no_e2e:
        del a32, b32
        torch.cuda.empty_cache()
        e2e = e2e_report(torch, nk, dev, A, B, max(4, args.steps // 2))
    extra = {}
    if not args.no_extra and rank == 0:
        extra["grouped_512_bf16"] = grouped_report(torch, nk, synth, dev)
        extra["conv_8x56x56x64_3x3"] = conv_report(torch, nk, synth, dev)
        rr = resnet_report(torch, synth, dev)
        if rr is not None:
            extra["resnet_stack_bf16"] = rr
        extra["grouped_conv_resnet_layers"] = grouped_conv_report(torch, nk, synth, dev)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    bf16_peak, _, src = peaks()
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "TFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": f"linalg.matmul precision sweep, BF16 in / FP32 accumulate, M=N=K={n}",
                   "inputs": "A, B ~ N(0,1) with 1% of entries x100 (SplitMix64 seed 3)",
                   "step": "cast A, cast+transpose B to BF16, tcgen05 GEMM (FP32 out), one nk_* call each",
                   "schedule": {"tile_m": sched[0], "tile_n": sched[1], "tile_k": sched[2], "cluster": sched[3],
                                "stages": sched[4], "split_k": sched[5]},
                   "l2": "inputs larger than L2 (268 MB FP32 per operand); no flush"},
        "roofline": {"bound": "tensor", "achieved": kern_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": kern_tflops / bf16_peak, "traffic": recorded_traffic("tc_gemm_bf16_8192"),
                     "kernel": "tc_gemm_kernel (BF16)", "peak_source": f"{src} bf16 burst (MEASURED_PEAKS.json)",
                     "algorithmic_flop_per_launch": flop},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        "e2e": e2e,
        "sweep": sweep,
        "accuracy": accuracy,
    }
    line.update(extra)
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(A, B, args.cpu_rows)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
