#!/usr/bin/env python
"""Benchmark: linalg.matmul precision sweep at M = N = K = 8192 on GB300.

One step is one pass of the whole BF16 hot path over synthetic operands
already resident in HBM: operand prep (FP32 -> BF16 casts, B transposed to
K-major) and the tcgen05 GEMM with its epilogue, all through the C ABI.
`value` is the useful FLOP rate of the whole step (2*M*N*K / step time); the
roofline object times the GEMM kernel alone with CUDA events on its stream.
The FP32 operands (268 MB each) exceed the 129 MB L2, so no flush is needed.

Beside the headline the line carries: the rest of the precision sweep (FP8,
BF16x3, FP32 and the ratios to FP32, with the FP8 peak measured on the box),
an end-to-end number through pinned host buffers with the copies inside the
timed region, the grouped-GEMM config (one persistent launch vs the same 512
GEMMs as separate calls, both replayed from CUDA graphs), the convolution
configs, the ResNet-style stack (schedules from the learned cost model vs
exhaustive search, and a chained forward whose layers feed each other), and
the FP64 oracle timed on the host's cores (all cores and one core).

Every configuration whose working set is smaller than L2 is timed three
ways: `warm` (the same buffers replayed back to back from a CUDA graph),
`flushed` (a 256 MiB buffer written before every call; the time of the
flushes alone is subtracted) and `rotating` (back-to-back calls cycling
through enough buffer sets that the inputs of each call were evicted by the
calls before it).  Rooflines use the flushed time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nk|reference]
  python bench.py --case CASE     one kernel family alone (the workloads the
                                  ncu summaries under profiles/ were taken on)

Under torchrun rank r computes row block r of one matmul whose A has
N x 8192 rows (B replicated; weak scaling: 8192 rows per rank).  rank 0
prints the line.  --impl reference times the FP64 CPU oracle alone.
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
FLUSH_BYTES = 256 << 20


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


# ------------------------------------------------------------------ CPU legs
def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return None


def _timed(fn, min_s=0.3):
    """Best-of wall time of fn() (repeated until min_s has passed, at least twice)."""
    fn()
    best, total, n = float("inf"), 0.0, 0
    while n < 2 or total < min_s:
        t0 = time.perf_counter()
        fn()
        dt = time.perf_counter() - t0
        best, total, n = min(best, dt), total + dt, n + 1
    return best


def cpu_legs(scale: float = 1.0) -> dict:
    """The FP64 oracle, as it stands, on each configuration (or a stated
    sample of it).  Operands are rounded to the precision's values and
    converted to FP64 before the clock starts: what is timed is the
    contraction (and the conv's padding and epilogue), not the conversion."""
    import oracle.nk_oracle as O
    from paper_2307_16080_gb300 import synth
    out = {}
    # FP32 matmul 256^3 (whole problem)
    A, B = synth.matmul_uniform(256, 256, 256)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    t = _timed(lambda: O.matmul(A64, B64))
    out["f32_matmul_256"] = {"tflops": 2 * 256 ** 3 / t / 1e12, "s": t, "sample": "whole problem"}
    # BF16 8192^3: a row sample of the bf16-rounded operands
    n = N_DEFAULT
    rows = max(8, int(128 * scale))
    A, B = synth.matmul_outlier(n, n, n, rows=(0, rows))
    Ar, Br = O.bf16_rn(A), O.bf16_rn(B)
    t = _timed(lambda: O.matmul(Ar, Br), min_s=1.0)
    out["bf16_matmul_8192"] = {"tflops": 2.0 * rows * n * n / t / 1e12, "s": t,
                               "sample": f"{rows} of {n} output rows, operands bf16-rounded before timing"}
    # FP32 conv 8x56x56x64 3x3 + bias + ReLU (whole problem)
    I, W, bias = synth.conv_resnet_block()
    I64, W64, b64 = I.astype(np.float64), W.astype(np.float64), bias.astype(np.float64)
    t = _timed(lambda: O.epilogue(O.conv2d_nhwc_hwcf(I64, W64, pad=(1, 1, 1, 1)), bias=b64, relu=True))
    f = 2.0 * 8 * 56 * 56 * 64 * 9 * 64
    out["f32_conv_8x56x56x64"] = {"tflops": f / t / 1e12, "s": t, "sample": "whole problem"}
    # grouped: the first groups of the 512
    shapes = synth.grouped_problems(512)
    G = max(4, int(48 * scale))
    As, Bs = synth.grouped_operands(shapes[:G])
    As = [O.bf16_rn(a) for a in As]
    Bs = [O.bf16_rn(b) for b in Bs]
    t = _timed(lambda: O.grouped_matmul(As, Bs))
    f = float(sum(2.0 * M * N * K for M, N, K in shapes[:G]))
    out["grouped_512_bf16"] = {"tflops": f / t / 1e12, "s": t, "sample": f"groups 0..{G - 1} of 512"}
    # the ResNet-style stack at batch 1 (whole stack, each layer on its own input)
    layers = []
    for li, L in enumerate(synth.resnet_stack(1)):
        x = O.bf16_rn(synth.half_normal(7, li, (L["N"], L["H"], L["W"], L["C"])))
        w = O.bf16_rn(synth.normal(7, 100 + li, (L["KH"], L["KW"], L["C"], L["F"]), 0.05))
        layers.append((x, w, L))

    def stack():
        for x, w, L in layers:
            O.conv2d_nhwc_hwcf(x, w, (L["stride"],) * 2, (1, 1), (L["pad"],) * 4)
    t = _timed(stack)
    f = sum(2.0 * L["N"] * ((L["H"] + 2 * L["pad"] - L["KH"]) // L["stride"] + 1) ** 2 * L["F"] * L["KH"] * L["KW"]
            * L["C"] for _, _, L in layers)
    out["resnet_stack_batch1_bf16"] = {"tflops": f / t / 1e12, "s": t, "sample": "whole stack, batch 1"}
    return out


def cpu_baseline(one_core: bool = True) -> dict:
    """cpu_legs() in fresh processes: once with the host's BLAS on every core,
    once pinned to a single core with one BLAS thread."""
    def run(env_extra, pin):
        env = dict(os.environ)
        env.update(env_extra)
        pre = (lambda: os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})) if pin else None
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-legs", "1.0" if not pin else "0.25"],
                           capture_output=True, text=True, env=env, preexec_fn=pre, timeout=600)
        if r.returncode:
            return {"error": r.stderr[-400:]}
        return json.loads(r.stdout.strip().splitlines()[-1])
    cores = len(os.sched_getaffinity(0))
    allc = run({}, False)
    res = {"cores": allc.pop("threads", None) or cores, "legs_all_cores": allc}
    if one_core:
        one = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
        o = run(one, True)
        o.pop("threads", None)
        res["legs_one_core"] = o
    return res


def run_cpu_legs(scale: float):
    out = cpu_legs(scale)
    out["threads"] = _blas_threads() or len(os.sched_getaffinity(0))
    print(json.dumps(out), flush=True)


def run_reference(args, rank):
    """The FP64 oracle on the headline workload: each step a sample of output
    rows of the BF16 8192^3 matmul on the bf16-rounded operands (rounded once,
    before the timed steps)."""
    if rank != 0:
        return
    import oracle.nk_oracle as O
    from paper_2307_16080_gb300 import synth
    n = args.n
    rows = args.ref_rows
    A, B = synth.matmul_outlier(n, n, n, rows=(0, rows))
    Ar, Br = O.bf16_rn(A), O.bf16_rn(B)
    for _ in range(min(args.warmup, 1)):
        O.matmul(Ar, Br)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.matmul(Ar, Br)
        times.append(time.perf_counter() - t0)
    flops = 2.0 * rows * n * n
    value = flops * len(times) / sum(times) / 1e12
    cores = _blas_threads() or len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"linalg.matmul precision sweep, BF16, M=N=K={n}; FP64 oracle on a sample"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{rows} of {n} output rows per step; operands bf16-rounded and "
                                       f"converted to FP64 once before the timed steps"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU timing
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


def _capture(torch, body):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        body()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            body()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    return g


def graph_time(torch, fn, calls=10, reps=10):
    """Warm device time of one call: `calls` back-to-back calls on the same
    buffers captured into a CUDA graph, replayed `reps` times between CUDA
    events.  The working set stays in L2 when it fits there."""
    def body():
        for _ in range(calls):
            fn()
    g = _capture(torch, body)
    return time_fn(torch, g.replay, reps) / calls


_FLUSH = {}


def flushed_time(torch, fn, calls=16, trials=5):
    """Cold-L2 device time of one call: a graph of `calls` x [write a 256 MiB
    buffer, call] minus a graph of `calls` x [write the buffer], median over
    `trials` pairs of replays.  Each call starts with none of its operands in
    L2."""
    dev = torch.cuda.current_device()
    if dev not in _FLUSH:
        _FLUSH[dev] = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    buf = _FLUSH[dev]

    def with_call():
        for _ in range(calls):
            buf.zero_()
            fn()

    def flush_only():
        for _ in range(calls):
            buf.zero_()
    g1 = _capture(torch, with_call)
    g0 = _capture(torch, flush_only)
    diffs = []
    for _ in range(trials):
        t1 = time_fn(torch, g1.replay, 2, warm=1)
        t0 = time_fn(torch, g0.replay, 2, warm=1)
        diffs.append((t1 - t0) / calls)
    return statistics.median(diffs)


def rotating_time(torch, make_call, set_bytes, reps=10, min_bytes=None):
    """Device time of one call with back-to-back calls that cycle through
    enough independent buffer sets (make_call(i) builds set i) that together
    they hold twice the L2: each call's inputs were evicted by the calls since
    its set was last used.  Returns (ms, sets)."""
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    need = min_bytes or 2 * l2
    sets = max(2, min(64, -(-need // max(1, int(set_bytes)))))
    calls = [make_call(i) for i in range(sets)]

    def body():
        for c in calls:
            c()
    g = _capture(torch, body)
    return time_fn(torch, g.replay, reps) / sets, sets


def timings3(torch, fn, make_call, set_bytes, calls=10):
    """warm, flushed and rotating times of one configuration (ms)."""
    w = graph_time(torch, fn, calls=calls, reps=10)
    f = flushed_time(torch, fn)
    r, sets = rotating_time(torch, make_call, set_bytes)
    return {"warm_ms": w, "flushed_ms": f, "rotating_ms": r, "rotating_sets": sets, "working_set_bytes": set_bytes}


# ------------------------------------------------------------------ reports
def fp8_peak(torch, dev, n=8192, sustain_s=3.0):
    """torch._scaled_mm on E4M3 operands at n^3 (cuBLASLt): burst (best of 10)
    and sustained (back to back for a few seconds) dense FP8 TFLOP/s."""
    try:
        a = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        bt = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        one = torch.ones((), device=dev)
        f = lambda: torch._scaled_mm(a, bt.t(), scale_a=one, scale_b=one, out_dtype=torch.bfloat16)  # noqa: E731
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        best = min(time_fn(torch, f, 1, warm=0) for _ in range(10))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(10, int(sustain_s / (best * 1e-3)))
        e0.record()
        for _ in range(k):
            f()
        e1.record()
        torch.cuda.synchronize()
        sus = e0.elapsed_time(e1) / k
        flop = 2.0 * n ** 3
        return {"burst_tflops": flop / (best * 1e-3) / 1e12, "sustained_tflops": flop / (sus * 1e-3) / 1e12,
                "how": f"torch._scaled_mm E4M3 x E4M3 -> BF16, {n}^3, best of 10 / {k} back to back"}
    except Exception as e:   # an older torch without _scaled_mm on this part
        return {"error": str(e)[:200]}


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
    329 GB/s together, so a step's 805 MB takes 2.45 ms at least."""
    n = A.shape[0]
    a_h = torch.from_numpy(A).pin_memory()
    b_h = torch.from_numpy(B).pin_memory()
    c_h = [torch.empty(A.shape[0], B.shape[1]).pin_memory() for _ in range(nbuf)]
    a32 = [torch.empty(n, B.shape[0], device=dev) for _ in range(nbuf)]
    b32 = [torch.empty(B.shape, device=dev) for _ in range(nbuf)]
    cc = [torch.empty(n, B.shape[1], device=dev) for _ in range(nbuf)]
    a16 = torch.empty(n, B.shape[0], dtype=torch.bfloat16, device=dev)
    bt16 = torch.empty(B.shape[1], B.shape[0], dtype=torch.bfloat16, device=dev)
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
    return {"value": 2.0 * n * B.shape[0] * B.shape[1] / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "h2d_bytes_per_step": (a_h.numel() + b_h.numel()) * 4, "d2h_bytes_per_step": c_h[0].numel() * 4,
            "how": f"host wall clock over pipelined steps (upload / compute / download streams, {nbuf} buffer sets)"}


def grouped_report(torch, nk, synth, dev):
    """512 uneven BF16 GEMMs: one persistent launch vs the same GEMMs as 512
    nk_matmul calls, both captured into CUDA graphs (device time)."""
    shapes = [tuple(int(v) for v in s) for s in synth.grouped_problems(512)]
    flop = float(sum(2.0 * M * N * K for (M, N, K) in shapes))
    set_bytes = sum(2 * M * K + 2 * N * K + 4 * M * N for (M, N, K) in shapes)

    def make_set(_i=0):
        a = [torch.empty(M, K, device=dev).uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in shapes]
        bt = [torch.empty(N, K, device=dev).uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in shapes]
        c = [torch.empty(M, N, device=dev) for (M, N, K) in shapes]
        return a, bt, c
    a, bt, c = make_set()
    groups, G = nk.make_groups(a, bt, c)
    from paper_2307_16080_gb300 import nk_tune as nt
    tuned, trep = nt.nk_grouped_tune(groups, G, reps=3)   # the autotuner picks the grouped tile
    plan = nk.nk_grouped_plan_create(groups, G, schedule=tuned)
    run = lambda: nk.nk_grouped_plan_run(plan)  # noqa: E731
    t_warm = graph_time(torch, run, calls=4, reps=10)
    t_flush = flushed_time(torch, run, calls=8)
    wss = [nk.workspace(nk.nk_matmul_workspace_size(a[g], bt[g].t(), c[g], "bf16"), dev) for g in range(G)]

    def per_gemm():
        for g in range(G):
            nk.nk_matmul(a[g], bt[g].t(), c[g], precision="bf16", ws=wss[g])
    t_calls = graph_time(torch, per_gemm, calls=1, reps=5)
    t_calls_flush = flushed_time(torch, per_gemm, calls=2, trials=3)
    t_eager = time_fn(torch, per_gemm, 3)
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)
    tf = lambda ms: flop / (ms * 1e-3) / 1e12  # noqa: E731
    return {"groups": G, "useful_flop": flop, "working_set_bytes": set_bytes,
            "persistent_warm_ms": t_warm, "persistent_flushed_ms": t_flush,
            "persistent_flushed_tflops": tf(t_flush), "persistent_warm_tflops": tf(t_warm),
            "per_gemm_graph_ms": t_calls, "per_gemm_graph_flushed_ms": t_calls_flush,
            "per_gemm_eager_ms": t_eager,
            "speedup_vs_per_gemm_graph": t_calls / t_warm,
            "speedup_vs_per_gemm_graph_flushed": t_calls_flush / t_flush,
            "speedup_vs_eager_calls": t_eager / t_warm,
            "frac_of_measured_bf16": tf(t_flush) / peaks()[0],
            "schedule": list(tuned), "tuned_ms": trep.best_ms, "untuned_default_ms": trep.default_ms,
            "schedules_timed": trep.timed,
            "how": "device time; per_gemm_graph = the 512 nk_matmul calls (built-in schedules) captured in one "
                   "CUDA graph; eager = the same calls issued from Python",
            "launches": {"persistent": 1, "per_gemm": G}}


def layer_roofline(N, H, W, C, F, KH, KW, stride, pad, ms, out_bytes=4, in_bytes=2, peak=None):
    """min(tensor peak, HBM x arithmetic intensity) for one conv layer:
    `in_bytes` per input element and per packed weight (2: BF16, 1: E4M3),
    `out_bytes` per output element (4: FP32, 2: BF16); achieved = FLOP /
    measured time.  peak: the dtype's dense tensor peak (default: BF16)."""
    bf16_peak, hbm, src = peaks()
    peak = peak or bf16_peak
    oh = (H + 2 * pad - KH) // stride + 1
    ow = (W + 2 * pad - KW) // stride + 1
    flop = 2.0 * N * oh * ow * F * KH * KW * C
    nbytes = float(in_bytes) * N * H * W * C + out_bytes * N * oh * ow * F + float(in_bytes) * KH * KW * C * F
    ai = flop / nbytes
    roof = min(peak, hbm * 1e-3 * ai)    # TFLOP/s
    achieved = flop / (ms * 1e-3) / 1e12
    return {"flop": flop, "bytes": nbytes, "ai_flop_per_byte": ai, "bound": "hbm" if roof < peak else "tensor",
            "roofline_tflops": roof, "achieved_tflops": achieved, "frac": achieved / roof,
            "peak_source": f"{src} (MEASURED_PEAKS.json; FP8: measured with torch._scaled_mm in this run)"}


def conv_layer_report(torch, nk, synth, dev, N, H=56, C=64, F=64, fp8_peak_tflops=None):
    """One 3x3 stride-1 layer N x H x H x C -> F (pad 1, bias + ReLU): FP32 on
    the CUDA cores; BF16 with a per-call weight cast and with packed weights
    (FP32 and BF16 output); E4M3 quantised per call from FP32 operands and
    from operands quantised once (FP32 and BF16 output).  Every variant
    warm / flushed / rotating; ratios to FP32 from the flushed times."""
    I, W, bias = synth.conv_resnet_block(N=N, H=H, W=H, C=C, F=F)
    i32, w32, b32 = (torch.from_numpy(x).to(dev) for x in (I, W, bias))
    flop = 2.0 * N * H * H * F * 9 * C
    pad = (1, 1, 1, 1)
    res = {"flop": flop, "shape": f"{N}x{H}x{H}x{C} -> {F}, 3x3, stride 1, pad 1, bias + ReLU"}
    o_elems = N * H * H * F

    def add(name, call_of, set_bytes, out_bytes=4, in_bytes=2, peak=None):
        t = timings3(torch, call_of(0), call_of, set_bytes)
        t["flushed_tflops"] = flop / (t["flushed_ms"] * 1e-3) / 1e12
        t["warm_tflops"] = flop / (t["warm_ms"] * 1e-3) / 1e12
        if in_bytes:
            t["roofline"] = layer_roofline(N, H, H, C, F, 3, 3, 1, 1, t["flushed_ms"], out_bytes, in_bytes, peak)
        res[name] = t

    def f32_call(i):
        ii = i32 if i == 0 else i32.clone()
        oo = torch.empty(N, H, H, F, device=dev)
        return lambda: nk.nk_conv2d_nhwc_hwcf(ii, w32, oo, pad=pad, bias=b32, relu=True)
    add("f32", f32_call, I.nbytes + o_elems * 4, in_bytes=0)
    i16 = i32.to(torch.bfloat16)
    wp = nk.nk_conv2d_pack_weights(w32)

    def bf16_call(packed, out_dtype=torch.float32):
        def make(i):
            ii = i16 if i == 0 else i16.clone()
            ww = (wp if i == 0 else nk.nk_conv2d_pack_weights(w32)) if packed else w32
            oo = torch.empty(N, H, H, F, device=dev, dtype=out_dtype)
            ws = nk.workspace(nk.nk_conv2d_workspace_size(ii, ww, oo, pad=pad, precision="bf16"), dev)
            return lambda: nk.nk_conv2d_nhwc_hwcf(ii, ww, oo, pad=pad, precision="bf16", bias=b32, relu=True, ws=ws)
        return make
    add("bf16_weight_cast_per_call", bf16_call(False), i16.numel() * 2 + o_elems * 4)
    add("bf16_packed", bf16_call(True), i16.numel() * 2 + o_elems * 4)
    add("bf16_packed_bf16_out", bf16_call(True, torch.bfloat16), i16.numel() * 2 + o_elems * 2, out_bytes=2)

    def fp8_call(i):
        ii = i32 if i == 0 else i32.clone()
        oo = torch.empty(N, H, H, F, device=dev)
        ws = nk.workspace(nk.nk_conv2d_workspace_size(ii, w32, oo, pad=pad, precision="fp8"), dev)
        return lambda: nk.nk_conv2d_nhwc_hwcf(ii, w32, oo, pad=pad, precision="fp8", bias=b32, relu=True, ws=ws)
    add("fp8_quantised_per_call", fp8_call, I.nbytes + o_elems * 4, in_bytes=0)
    wq, sw = nk.nk_conv2d_pack_weights_fp8(w32)
    iq, si = nk.quantize_nhwc_fp8(i32)
    s_i, s_w = float(si.item()), float(sw.item())

    def fp8q_call(out_dtype):
        def make(i):
            qi = iq if i == 0 else iq.clone()
            qw = wq if i == 0 else nk.nk_conv2d_pack_weights_fp8(w32)[0]
            oo = torch.empty(N, H, H, F, device=dev, dtype=out_dtype)
            ws = nk.workspace(nk.nk_conv2d_workspace_size(qi, qw, oo, pad=pad, precision="fp8"), dev)
            return lambda: nk.nk_conv2d_nhwc_hwcf(qi, qw, oo, pad=pad, precision="fp8", bias=b32, relu=True, ws=ws,
                                                  scale_i=s_i, scale_w=s_w)
        return make
    add("fp8_prequantised", fp8q_call(torch.float32), iq.numel() + o_elems * 4, in_bytes=1, peak=fp8_peak_tflops)
    add("fp8_prequantised_bf16_out", fp8q_call(torch.bfloat16), iq.numel() + o_elems * 2, out_bytes=2, in_bytes=1,
        peak=fp8_peak_tflops)
    nk.nk_sync_status()
    f32 = res["f32"]["flushed_ms"]
    res["ratios_flushed_vs_f32"] = {k: f32 / v["flushed_ms"] for k, v in res.items()
                                    if isinstance(v, dict) and "flushed_ms" in v and k != "f32"}
    res["ratios_warm_vs_f32"] = {k: res["f32"]["warm_ms"] / v["warm_ms"] for k, v in res.items()
                                 if isinstance(v, dict) and "warm_ms" in v and k != "f32"}
    return res


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
        tot["tuner_timing"] = nt.timing_method()
        tot["stack_graph"] = stack_graph(torch, synth, dev, b, picks, tot["flop"])
        tot["model_picks"] = [[int(v) for v in pk] for pk in picks]   # schedule tuples, one per layer
        out[f"batch{b}"] = tot
    nt.nk_tune_release()
    return out


def stack_roofline_ms(synth, batch, out_bytes=4):
    """Sum over the 20 layers of each layer's roofline time; out_bytes is one
    value for every layer or a list with one per layer."""
    roof_ms = 0.0
    for li, L in enumerate(synth.resnet_stack(batch)):
        ob = out_bytes[li] if isinstance(out_bytes, (list, tuple)) else out_bytes
        r = layer_roofline(L["N"], L["H"], L["W"], L["C"], L["F"], L["KH"], L["KW"], L["stride"], L["pad"], 1.0,
                           ob)
        roof_ms += r["flop"] / (r["roofline_tflops"] * 1e12) * 1e3
    return roof_ms


def stack_graph(torch, synth, dev, batch, picks, flop):
    """The 20 stack layers through the public API, each on its own BF16
    input (packed BF16 weights, bias + ReLU, the cost model's pick as
    schedule, FP32 output), all 20 captured into one CUDA graph."""
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
    ms_flushed = flushed_time(torch, forward, calls=4, trials=3)
    nk.nk_set_pdl(False)   # the same graph captured with plain stream ordering between kernels
    ms_serial = graph_time(torch, forward, calls=2, reps=10)
    nk.nk_set_pdl(True)
    nk.nk_sync_status()
    kernels = sum(2 if sched[5] > 1 else 1 for sched in picks)   # split-K adds its reduce
    roof_ms = stack_roofline_ms(synth, batch)
    return {"warm_ms": ms, "flushed_ms": ms_flushed, "tflops_flushed": flop / (ms_flushed * 1e-3) / 1e12,
            "kernels_per_forward": kernels, "warm_ms_without_pdl": ms_serial, "pdl_speedup": ms_serial / ms,
            "roofline_ms": roof_ms, "frac_of_roofline_flushed": roof_ms / ms_flushed,
            "how": "20 independent nk_conv2d calls on packed BF16 weights in one CUDA graph, device time; "
                   "flushed: 256 MiB written before each forward, flush time subtracted"}


def chained_forward_report(torch, nk, synth, dev, picks=None):
    """The ResNet-style stack as a real forward: every 3x3 s1 layer reads the
    BF16 output its predecessor wrote (bias + ReLU fused, rounded to BF16 in
    the epilogue); each stage's stride-2 3x3 and 1x1 projection read the
    stage input, and the stage's last conv adds the projection (a fused ADD
    of the residual) before its ReLU.  One CUDA graph per batch, with the
    built-in schedules and, when given (picks[batch]: one per layer), with
    the cost model's top-5 picks of the stack report."""
    import paper_2307_16080_gb300.forward as fwd
    out = {}
    for b in (1, 8, 32):
        rec = {}
        runs = [("default", None)]
        if picks and picks.get(b):
            runs.append(("model", [tuple(pk) for pk in picks[b]]))
        for name, scheds in runs:
            net = fwd.ResNetStack(b, dev, seed=5, schedules=scheds)
            x = torch.empty(b, 56, 56, 64, device=dev).uniform_(0, 1).to(torch.bfloat16)
            net.bind(x)
            ms = graph_time(torch, net.run, calls=2, reps=10)
            ms_flushed = flushed_time(torch, net.run, calls=4, trials=3)
            nk.nk_sync_status()
            # BF16 activations; the projections and the head write FP32
            ob = [4 if net.role(li) in ("projection", "head") else 2 for li in range(20)]
            roof_ms = stack_roofline_ms(synth, b, out_bytes=ob)
            r = {"warm_ms": ms, "flushed_ms": ms_flushed, "tflops_flushed": net.flop / (ms_flushed * 1e-3) / 1e12,
                 "roofline_ms": roof_ms, "frac_of_roofline_flushed": roof_ms / ms_flushed,
                 "kernels_per_forward": net.kernels}
            if name == "default":
                rec.update(r)
            else:
                rec["model_schedules"] = r
        out[f"batch{b}"] = rec
    return out


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
    run = lambda: nk.nk_grouped_plan_run(plan)  # noqa: E731
    t_grouped = graph_time(torch, run, calls=2, reps=10)
    t_grouped_f = flushed_time(torch, run, calls=4, trials=3)
    wss = [nk.workspace(nk.nk_conv2d_workspace_size(d["I"], d["W"], d["O"], d["stride"], (1, 1), d["pad"], "bf16"),
                        dev) for d in convs]

    def separate():
        for d, ws in zip(convs, wss):
            nk.nk_conv2d_nhwc_hwcf(d["I"], d["W"], d["O"], d["stride"], (1, 1), d["pad"], "bf16", bias=d["bias"],
                                   relu=True, ws=ws)
    t_sep = graph_time(torch, separate, calls=2, reps=10)
    t_sep_f = flushed_time(torch, separate, calls=4, trials=3)
    nk.nk_grouped_plan_destroy(plan)
    nk.nk_sync_status()
    return {"groups": G, "batch": batch, "flop": flop, "one_launch_warm_ms": t_grouped,
            "one_launch_flushed_ms": t_grouped_f, "one_launch_flushed_tflops": flop / (t_grouped_f * 1e-3) / 1e12,
            "separate_warm_ms": t_sep, "separate_flushed_ms": t_sep_f,
            "speedup_warm": t_sep / t_grouped, "speedup_flushed": t_sep_f / t_grouped_f,
            "schedule": list(tuned), "schedules_timed": trep.timed, "untuned_default_ms": trep.default_ms,
            "how": "device time of CUDA-graph replays; grouped: per-tap kernel, tile from nk_conv2d_grouped_tune"}


def sharded_extras(torch, nk, synth, dev, world, rank):
    """Under torchrun: the other two splits of the path, each rank on its own
    device memory with no data-path collective.  The 512-group GEMM by LPT
    over ranks on the cost model's predicted time of each group, and the
    32 x 56 x 56 x 64 conv by blocks of images.  Time = max over ranks."""
    from paper_2307_16080_gb300 import costmodel, shard
    from paper_2307_16080_gb300 import nk_tune as nt
    out = {}
    shapes = [tuple(int(v) for v in s) for s in synth.grouped_problems(512)]
    probs = [nt.matmul_problem(M, N, K, "bf16") for (M, N, K) in shapes]
    if os.path.exists(costmodel.MODEL_PATH):
        P, ym, ys = costmodel.load_model()
        cost, how = costmodel.predicted_ms(P, ym, ys, probs), "cost-model prediction of each group's time"
    else:
        cost, how = shard.gemm_flops(shapes), "2*M*N*K"
    owner, loads = shard.lpt_assign(cost, world)
    mine = [shapes[g] for g in shard.groups_of_rank(owner, rank)]
    a = [torch.empty(M, K, device=dev).uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in mine]
    bt = [torch.empty(N, K, device=dev).uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in mine]
    c = [torch.empty(M, N, device=dev) for (M, N, K) in mine]
    groups, G = nk.make_groups(a, bt, c)
    plan = nk.nk_grouped_plan_create(groups, G)
    t = flushed_time(torch, lambda: nk.nk_grouped_plan_run(plan), calls=8)
    nk.nk_grouped_plan_destroy(plan)
    t_max = shard.max_over_ranks(t)
    flop = float(sum(2.0 * M * N * K for (M, N, K) in shapes))
    out["grouped_512_lpt"] = {"ms_max_over_ranks": t_max, "tflops_all_ranks": flop / (t_max * 1e-3) / 1e12,
                              "predicted_load_max_over_mean": float(loads.max() / loads.mean()), "cost": how}
    Nb = 32
    n0, n1 = shard.batch_blocks(Nb, world)[rank]
    I, W, bias = synth.conv_resnet_block(N=Nb)
    i16 = torch.from_numpy(I[n0:n1]).to(dev).to(torch.bfloat16)
    wp = nk.nk_conv2d_pack_weights(torch.from_numpy(W).to(dev))
    b = torch.from_numpy(bias).to(dev)
    o = torch.empty(n1 - n0, 56, 56, 64, device=dev)
    t = flushed_time(torch, lambda: nk.nk_conv2d_nhwc_hwcf(i16, wp, o, pad=(1, 1, 1, 1), precision="bf16", bias=b,
                                                           relu=True)) if n1 > n0 else 0.0
    t_max = shard.max_over_ranks(t)
    out["conv_32x56x56x64_by_batch"] = {"ms_max_over_ranks": t_max, "images_per_rank": n1 - n0,
                                        "tflops_all_ranks": 2.0 * Nb * 56 * 56 * 64 * 576 / (t_max * 1e-3) / 1e12}
    nk.nk_sync_status()
    return out


# ------------------------------------------------------------------ --case
def _case_emit(name, ms, bytes_=None, flop=None, **kw):
    bf16, hbm, _ = peaks()
    out = {"case": name, "ms": ms}
    if bytes_ is not None:
        gbs = bytes_ / (ms * 1e-3) / 1e9
        out.update({"algorithmic_bytes": bytes_, "GB/s": gbs, "frac_of_measured_hbm": gbs / hbm})
    if flop is not None:
        tf = flop / (ms * 1e-3) / 1e12
        out.update({"flop": flop, "TFLOP/s": tf, "frac_of_measured_bf16": tf / bf16})
    out.update(kw)
    print(json.dumps(out), flush=True)


def run_case(name, reps, schedule=None, shape=None):
    """One kernel family alone, on a fixed workload (device times of CUDA
    graph replays; the inputs of each are larger than L2, or the timing is
    the flushed one).  schedule: a fixed tile for the grouped case instead
    of its tuner (so a profiler sees the measured kernel first), or for the
    conv cases instead of the built-in choice; shape: N,H,C,F of the conv
    cases (3x3, stride 1, pad 1, H x H images)."""
    import torch

    import paper_2307_16080_gb300.nk as nk
    from paper_2307_16080_gb300 import synth
    torch.cuda.set_device(0)
    nk.lib()
    n = 8192
    if name == "cast":
        x = torch.randn(n, n, device="cuda")
        y = torch.empty(n, n, dtype=torch.bfloat16, device="cuda")
        _case_emit("cast_rows bf16 8192^2", graph_time(torch, lambda: nk.nk_cast_bf16(x, y), 4, reps),
                   bytes_=n * n * 6)
        _case_emit("cast_transpose bf16 8192^2",
                   graph_time(torch, lambda: nk.nk_cast_bf16(x, y, transpose=True), 4, reps), bytes_=n * n * 6)
    elif name == "amax":
        x = torch.randn(n, n, device="cuda")
        a = torch.empty(1, device="cuda")
        ws = nk.workspace(nk.lib().nk_prep_workspace_size(n * n))
        _case_emit("amax 8192^2", graph_time(torch, lambda: nk.nk_amax(x, a, ws), 4, reps), bytes_=n * n * 4)
    elif name == "direct":
        for batch in (1, 16):
            i = torch.randn(batch, 1, 1280, 1280, device="cuda")
            k = torch.randn(3, 1, 3, 3, device="cuda")
            o = torch.empty(batch, 3, 1278, 1278, device="cuda")
            b = batch * (1280 * 1280 + 3 * 1278 * 1278) * 4
            f = 2.0 * batch * 3 * 1278 * 1278 * 9
            call = lambda: nk.nk_conv2d_nchw_fchw(i, k, o)  # noqa: E731
            ms = flushed_time(torch, call) if batch == 1 else graph_time(torch, call, 4, reps)
            _case_emit(f"direct nchw conv ({batch},1,1280,1280) Co=3 3x3", ms, bytes_=b, flop=f,
                       timing="flushed" if batch == 1 else "inputs larger than L2")
    elif name in ("conv", "conv_window", "conv_tap", "conv8"):
        N, H, C, F = 8 if name == "conv8" else 32, 56, 64, 64
        if shape is not None:
            N, H, C, F = shape
        sched = {"conv": None, "conv8": None, "conv_window": (128, 64, 64 * 9, 1, 1, 1),
                 "conv_tap": (128, 64, 64, 1, 3, 1)}[name]
        sched = schedule if schedule is not None else sched
        i = torch.randn(N, H, H, C, device="cuda").abs().to(torch.bfloat16)
        w = nk.nk_conv2d_pack_weights(torch.randn(3, 3, C, F, device="cuda") * (2.0 / (9 * C)) ** 0.5)
        o = torch.empty(N, H, H, F, device="cuda")
        ws = nk.workspace(nk.nk_conv2d_workspace_size(i, w, o, pad=(1, 1, 1, 1), precision="bf16", schedule=sched))
        call = lambda: nk.nk_conv2d_nhwc_hwcf(i, w, o, pad=(1, 1, 1, 1), precision="bf16",  # noqa: E731
                                              schedule=sched, ws=ws)
        f = 2.0 * N * H * H * F * 9 * C
        b = N * H * H * (C * 2 + F * 4) + 9 * C * F * 2
        _case_emit(f"bf16 conv {N}x{H}x{H}x{C} -> {F} 3x3 ({name})", flushed_time(torch, call), bytes_=b, flop=f,
                   timing="flushed", warm_ms=graph_time(torch, call, 10, reps),
                   schedule=list(sched) if sched is not None else None)
    elif name == "stack8":
        calls, flop = [], 0.0
        for L in synth.resnet_stack(8):
            oh = (L["H"] + 2 * L["pad"] - L["KH"]) // L["stride"] + 1
            x = torch.randn(L["N"], L["H"], L["W"], L["C"], device="cuda").abs().to(torch.bfloat16)
            w = nk.nk_conv2d_pack_weights(torch.randn(L["KH"], L["KW"], L["C"], L["F"], device="cuda") * 0.05)
            bb = torch.randn(L["F"], device="cuda") * 0.1
            o = torch.empty(L["N"], oh, oh, L["F"], device="cuda")
            st, pd = (L["stride"],) * 2, (L["pad"],) * 4
            ws = nk.workspace(nk.nk_conv2d_workspace_size(x, w, o, st, (1, 1), pd, "bf16"))
            calls.append((x, w, o, st, pd, bb, ws))
            flop += 2.0 * L["N"] * oh * oh * L["F"] * L["KH"] * L["KW"] * L["C"]

        def forward():
            for (x, w, o, st, pd, bb, ws) in calls:
                nk.nk_conv2d_nhwc_hwcf(x, w, o, st, (1, 1), pd, "bf16", bias=bb, relu=True, ws=ws)
        _case_emit("resnet stack batch 8, 20 convs (built-in schedules)", flushed_time(torch, forward, 4, 3),
                   flop=flop, timing="flushed")
    elif name in ("chain8", "chain32"):
        import paper_2307_16080_gb300.forward as fwd
        nb = 8 if name == "chain8" else 32
        net = fwd.ResNetStack(nb, "cuda", seed=5)
        x = torch.empty(nb, 56, 56, 64, device="cuda").uniform_(0, 1).to(torch.bfloat16)
        net.bind(x)
        _case_emit(f"chained resnet forward batch {nb} (BF16 activations)", flushed_time(torch, net.run, 4, 3),
                   flop=net.flop, timing="flushed")
    elif name == "conv_fp8":
        # E4M3 stacked window kernel on pre-quantised operands, 32 x 14 x 14 x 256 3x3
        N, H, C, F = 32, 14, 256, 256
        i32 = torch.randn(N, H, H, C, device="cuda").abs()
        w32 = torch.randn(3, 3, C, F, device="cuda") * 0.03
        iq, si = nk.quantize_nhwc_fp8(i32)
        wq, sw = nk.nk_conv2d_pack_weights_fp8(w32)
        o = torch.empty(N, H, H, F, device="cuda")
        ws = nk.workspace(nk.nk_conv2d_workspace_size(iq, wq, o, pad=(1, 1, 1, 1), precision="fp8"))
        s_i, s_w = float(si.item()), float(sw.item())
        call = lambda: nk.nk_conv2d_nhwc_hwcf(iq, wq, o, pad=(1, 1, 1, 1), precision="fp8",  # noqa: E731
                                              relu=True, ws=ws, scale_i=s_i, scale_w=s_w)
        f = 2.0 * N * H * H * F * 9 * C
        b = N * H * H * (C + F * 4) + 9 * C * F
        _case_emit(f"fp8 conv {N}x{H}x{H}x{C} -> {F} 3x3, pre-quantised", flushed_time(torch, call), bytes_=b,
                   flop=f, timing="flushed", warm_ms=graph_time(torch, call, 10, reps))
    elif name == "grouped":
        shapes = [tuple(int(v) for v in s) for s in synth.grouped_problems(512)]
        a = [torch.empty(M, K, device="cuda").uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in shapes]
        bt = [torch.empty(N, K, device="cuda").uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in shapes]
        c = [torch.empty(M, N, device="cuda") for (M, N, K) in shapes]
        groups, G = nk.make_groups(a, bt, c)
        from paper_2307_16080_gb300 import nk_tune as nt
        best = schedule if schedule is not None else nt.nk_grouped_tune(groups, G, reps=3)[0]
        plan = nk.nk_grouped_plan_create(groups, G, schedule=best)
        f = float(sum(2.0 * M * N * K for (M, N, K) in shapes))
        _case_emit("grouped 512 bf16 gemms", flushed_time(torch, lambda: nk.nk_grouped_plan_run(plan), 8), flop=f,
                   timing="flushed", schedule=list(best))
        nk.nk_grouped_plan_destroy(plan)
    elif name == "splitk":
        M, N, K, s = 1024, 1024, 16384, 8
        a = torch.randn(M, K, device="cuda")
        b = torch.randn(K, N, device="cuda")
        c = torch.empty(M, N, device="cuda")
        sched = (64, 64, 16, 1, 2, s)
        ws = nk.workspace(nk.nk_matmul_workspace_size(a, b, c, "f32", sched))
        _case_emit("f32 split-K 8 1024x1024x16384", graph_time(
            torch, lambda: nk.nk_matmul(a, b, c, precision="f32", schedule=sched, ws=ws), 4, reps),
            flop=2.0 * M * N * K, timing="inputs larger than L2")
    elif name == "gemm":
        A, B = synth.matmul_outlier(n, n, n)
        a16 = torch.from_numpy(A).cuda().to(torch.bfloat16)
        bt16 = torch.from_numpy(B).cuda().t().contiguous().to(torch.bfloat16)
        c = torch.empty(n, n, device="cuda")
        ws = nk.workspace(nk.nk_matmul_workspace_size(a16, bt16.t(), c, "bf16"))
        _case_emit("bf16 gemm 8192^3", time_fn(torch, lambda: nk.nk_matmul(a16, bt16.t(), c, precision="bf16",
                                                                            ws=ws), reps),
                   flop=2.0 * n ** 3, timing="inputs larger than L2")
    else:
        raise SystemExit(f"unknown case {name}")
    nk.nk_sync_status()


CASES = ("cast", "amax", "direct", "conv", "conv8", "conv_window", "conv_tap", "conv_fp8", "stack8", "chain8",
         "chain32", "grouped", "splitk", "gemm")


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nk", choices=["nk", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--ref-rows", type=int, default=128)
    ap.add_argument("--case", choices=CASES, help="time one kernel family alone and exit")
    ap.add_argument("--reps", type=int, default=20, help="replays per --case timing")
    ap.add_argument("--schedule", default=None,
                    help="--case grouped / conv*: fixed tile_m,tile_n,tile_k,cluster,stages,split_k")
    ap.add_argument("--shape", default=None, help="--case conv*: N,H,C,F of a 3x3 stride-1 layer")
    ap.add_argument("--cpu-legs", type=float, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-sweep", action="store_true", help="skip the FP8/BF16x3/FP32 sweep")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-check", action="store_true", help="skip the sampled accuracy check")
    ap.add_argument("--no-extra", action="store_true", help="skip the grouped / conv / ResNet reports")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.cpu_legs is not None:
        run_cpu_legs(args.cpu_legs)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.case:
        run_case(args.case, args.reps,
                 tuple(int(v) for v in args.schedule.split(",")) if args.schedule else None,
                 tuple(int(v) for v in args.shape.split(",")) if args.shape else None)
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
    # Row block `rank` of one matmul with world * n rows (B replicated):
    # every rank computes n x n x n, so per-GPU work is fixed as N grows.
    M_all = n * world
    r0, r1 = shard.row_blocks(M_all, world)[rank]
    A, B = synth.matmul_outlier(M_all, n, n, rows=(r0, r1))
    m = r1 - r0
    a32 = torch.from_numpy(A).to(dev)
    b32 = torch.from_numpy(B).to(dev)
    c = torch.empty(m, n, device=dev)
    a16 = torch.empty(m, n, dtype=torch.bfloat16, device=dev)
    bt16 = torch.empty(n, n, dtype=torch.bfloat16, device=dev)   # B^T, K-major
    st = torch.cuda.current_stream()
    ws = nk.workspace(nk.nk_matmul_workspace_size(a16, bt16.t(), c, "bf16"), dev)
    sched = nt.nk_default_schedule(nt.matmul_problem(m, n, n, "bf16"))

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
    flop = 2.0 * m * n * n
    value = 2.0 * M_all * n * n * args.steps / (ms * 1e-3) / 1e12
    kern_tflops = flop / (kern_ms * 1e-3) / 1e12

    accuracy = {}
    if rank == 0 and not args.no_check:
        import oracle.nk_oracle as O
        rows = np.sort(synth.raw_u64(77, 1, 512) % np.uint64(m)).astype(np.int64)
        rows = np.unique(rows)
        got = c[torch.from_numpy(rows).to(dev)].cpu().numpy()
        Br = O.bf16_rn(B)
        accuracy["err_vs_bf16_inputs_sampled"] = O.rel_frobenius(got, O.matmul(O.bf16_rn(A[rows]), Br))
        accuracy["err_vs_fp32_inputs_sampled"] = O.rel_frobenius(got, O.matmul(A[rows], B))
        accuracy["rows"] = int(len(rows))
        accuracy["bounds"] = {"vs_bf16_inputs": 1e-5, "vs_fp32_inputs": 8e-3}

    sweep = None if args.no_sweep else sweep_report(torch, nk, dev, a32, b32, c, flop, kern_tflops)
    # the FP8 peak after the sweep: its seconds-long loop would otherwise leave
    # the sweep's kernels to run on a GPU still at its power limit
    fp8pk = fp8_peak(torch, dev) if (rank == 0 and not args.no_sweep) else {}
    if sweep is not None and "burst_tflops" in fp8pk:
        sweep["fp8_frac_of_measured_fp8_burst"] = sweep["fp8"] / fp8pk["burst_tflops"]
    e2e = None
    if not args.no_e2e:
        del a32, b32
        torch.cuda.empty_cache()
        e2e = e2e_report(torch, nk, dev, A, B, max(4, args.steps // 2))
        e2e["value"] = e2e["value"] * world   # every rank moves and computes its own block
    extra = {}
    if not args.no_extra and world == 1:   # under torchrun the line carries the sharded extras instead
        extra["grouped_512_bf16"] = grouped_report(torch, nk, synth, dev)
        fp8t = fp8pk.get("burst_tflops")
        extra["conv_8x56x56x64_3x3"] = conv_layer_report(torch, nk, synth, dev, 8, fp8_peak_tflops=fp8t)
        extra["conv_32x56x56x64_3x3"] = conv_layer_report(torch, nk, synth, dev, 32, fp8_peak_tflops=fp8t)
        extra["conv_8x28x28x128_3x3"] = conv_layer_report(torch, nk, synth, dev, 8, 28, 128, 128, fp8t)
        extra["conv_32x14x14x256_3x3"] = conv_layer_report(torch, nk, synth, dev, 32, 14, 256, 256, fp8t)
        rr = resnet_report(torch, synth, dev)
        if rr is not None:
            extra["resnet_stack_bf16"] = rr
        picks = {b: rr[f"batch{b}"]["model_picks"] for b in (1, 8, 32)} if rr is not None else None
        extra["resnet_chained_forward_bf16"] = chained_forward_report(torch, nk, synth, dev, picks)
        extra["grouped_conv_resnet_layers"] = grouped_conv_report(torch, nk, synth, dev)
        extra["fp8_peak_measured"] = fp8pk

    if world > 1 and not args.no_extra:
        extra["sharded"] = sharded_extras(torch, nk, synth, dev, world, rank)
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
        "config": {"workload": f"linalg.matmul precision sweep, BF16 in / FP32 accumulate, M=N=K={n} per GPU",
                   "inputs": "A, B ~ N(0,1) with 1% of entries x100 (SplitMix64 seed 3)",
                   "step": "cast A, cast+transpose B to BF16, tcgen05 GEMM (FP32 out), one nk_* call each",
                   "sharding": f"row blocks of one {M_all} x {n} A over {world} GPU(s), B replicated, "
                               "no data-path collective",
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
        cb = cpu_baseline()
        leg = cb["legs_all_cores"].get("bf16_matmul_8192", {})
        line["cpu_baseline"] = {"value": leg.get("tflops"), "unit": "TFLOP/s", "cores": cb["cores"], "kind": "oracle",
                                "sample": leg.get("sample", "") + " (BF16 8192^3 workload; FP64 contraction only)",
                                "legs": cb}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
