#!/usr/bin/env python
"""Benchmark: linalg.matmul precision sweep at M = N = K = 8192 on one GB300.

One step is one pass of the whole BF16 hot path over the synthetic operands:
operand prep (FP32 -> BF16 casts, B transposed to K-major) followed by the
tcgen05 GEMM with its epilogue, all through the C ABI.  `value` is the useful
FLOP rate of the whole step (2*M*N*K / step time); the roofline object times
the GEMM kernel alone with CUDA events on its stream.  Inputs (268 MB per
FP32 operand) are larger than the 129 MB L2, so no flush is needed between
steps.  FP32, BF16x3 and FP8 GEMM throughputs of the same sweep are reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nk|reference]

With --impl reference the FP64 CPU oracle is timed on a bounded sample of
the same workload (rank 0 only).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 8192
METRIC = "TFLOP/s & % of tensor peak, matmul/conv2d, BF16/FP8 vs FP32 at stated error"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), float(p["hbm_gbs"]), "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


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
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


def cpu_baseline(A, B, rows: int):
    """The FP64 oracle (as it stands) on a sample of `rows` rows of the BF16 workload."""
    import oracle.nk_oracle as O
    t0 = time.perf_counter()
    O.matmul_precision(A[:rows], B, "bf16")
    dt = time.perf_counter() - t0
    flops = 2.0 * rows * B.shape[0] * B.shape[1]
    try:
        from threadpoolctl import threadpool_info
        cores = max(int(i.get("num_threads", 1)) for i in threadpool_info()) if threadpool_info() else 1
    except Exception:
        cores = len(os.sched_getaffinity(0))
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"{rows} of {A.shape[0]} output rows of the BF16 8192^3 matmul "
                      f"(bf16 rounding + FP64 numpy matmul), {dt:.1f} s"}


def run_reference(args, rank):
    if rank != 0:
        return
    from paper_2307_16080_gb300 import synth
    n = args.n
    A, B = synth.matmul_outlier(n, n, n)
    rows = args.ref_rows
    for _ in range(args.warmup):
        pass
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        import oracle.nk_oracle as O
        O.matmul_precision(A[:rows], B, "bf16")
        times.append(time.perf_counter() - t0)
    flops = 2.0 * rows * n * n
    value = flops * len(times) / sum(times) / 1e12
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"linalg.matmul bf16 {n}x{n}x{n} (precision sweep), oracle sample"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{rows} output rows per step"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    from paper_2307_16080_gb300 import synth

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    n = args.n
    A, B = synth.matmul_outlier(n, n, n)            # same problem on every rank (weak scaling)
    a32 = torch.from_numpy(A).to(dev)
    b32 = torch.from_numpy(B).to(dev)
    c = torch.empty(n, n, device=dev)
    a16 = torch.empty(n, n, dtype=torch.bfloat16, device=dev)
    bt16 = torch.empty(n, n, dtype=torch.bfloat16, device=dev)   # B^T, K-major
    st = torch.cuda.current_stream()
    ws = nk.workspace(nk.nk_matmul_workspace_size(a16, bt16.t(), c, "bf16"), dev)

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
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(st)
    for i in range(args.steps):
        step(kev[i])
    e1.record(st)
    barrier()
    clk = clocks.stop()
    nk.nk_sync_status()
    ms = e0.elapsed_time(e1)
    kern_ms = sum(a.elapsed_time(b) for a, b in kev) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    flop = 2.0 * n * n * n
    value = flop * args.steps * world / (ms * 1e-3) / 1e12
    ms_step = ms / args.steps

    # accuracy of this run's output on sampled rows (device FP64 norm vs host oracle rows)
    extra = {}
    if rank == 0 and not args.no_check:
        import oracle.nk_oracle as O
        rows = np.sort(synth.raw_u64(77, 1, 32) % np.uint64(n)).astype(np.int64)
        got = c[torch.from_numpy(rows).to(dev)].cpu().numpy()
        extra["err_vs_bf16_inputs_sampled"] = O.rel_frobenius(got, O.matmul(O.bf16_rn(A[rows]), O.bf16_rn(B)))
        extra["err_vs_fp32_inputs_sampled"] = O.rel_frobenius(got, O.matmul(A[rows], B))

    # precision sweep: GEMM kernel time per precision (operands already prepared)
    sweep = {}
    if not args.no_sweep:
        def time_it(fn, reps):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(st)
            for _ in range(reps):
                fn()
            s1.record(st)
            torch.cuda.synchronize()
            return s0.elapsed_time(s1) / reps
        sweep["bf16"] = flop / (kern_ms * 1e-3) / 1e12
        amax = torch.empty(2, device=dev)
        nk.nk_amax(a32, amax[0:1])
        nk.nk_amax(b32, amax[1:2])
        sc = torch.empty(2, device=dev)
        a8 = torch.empty(n, n, dtype=torch.uint8, device=dev)
        bt8 = torch.empty(n, n, dtype=torch.uint8, device=dev)
        nk.nk_cast_fp8(a32, amax[0:1], a8, scale_out=sc[0:1])
        nk.nk_cast_fp8(b32, amax[1:2], bt8, transpose=True, scale_out=sc[1:2])
        torch.cuda.synchronize()
        sa, sb = float(sc[0].item()), float(sc[1].item())
        ws8 = nk.workspace(nk.nk_matmul_workspace_size(a8, bt8.t(), c, "fp8"), dev)
        t8 = time_it(lambda: nk.nk_matmul(a8, bt8.t(), c, precision="fp8", scale_a=sa, scale_b=sb, ws=ws8), 10)
        sweep["fp8"] = flop / (t8 * 1e-3) / 1e12
        del a8, bt8
        wsx = nk.workspace(nk.nk_matmul_workspace_size(a32, b32, c, "bf16x3"), dev)
        tx = time_it(lambda: nk.nk_matmul(a32, b32, c, precision="bf16x3", ws=wsx), 5)
        sweep["bf16x3_with_prep"] = flop / (tx * 1e-3) / 1e12
        del wsx
        wsf = nk.workspace(nk.nk_matmul_workspace_size(a32, b32, c, "f32"), dev)
        tf = time_it(lambda: nk.nk_matmul(a32, b32, c, precision="f32", ws=wsf), 2)
        sweep["f32"] = flop / (tf * 1e-3) / 1e12
        sweep["bf16_over_f32"] = sweep["bf16"] / sweep["f32"]
        sweep["fp8_over_f32"] = sweep["fp8"] / sweep["f32"]
        sweep["unit"] = "TFLOP/s (GEMM kernel; bf16x3 includes its split pass)"
        nk.nk_sync_status()

    # end to end through the public API: pinned host FP32 in, host FP32 C out
    e2e = None
    if not args.no_e2e:
        a_h = torch.from_numpy(A).pin_memory()
        b_h = torch.from_numpy(B).pin_memory()
        c_h = torch.empty(n, n).pin_memory()

        def e2e_step():
            a32.copy_(a_h, non_blocking=True)
            b32.copy_(b_h, non_blocking=True)
            step()
            c_h.copy_(c, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        e2e_reps = max(3, args.steps // 4)
        barrier()
        t0 = time.perf_counter()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(st)
        for _ in range(e2e_reps):
            e2e_step()
        f1.record(st)
        barrier()
        e2e_ms = max(f0.elapsed_time(f1), (time.perf_counter() - t0) * 1e3) / e2e_reps
        nk.nk_sync_status()
        e2e = {"value": flop / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 2 * n * n * 4, "d2h_bytes_per_step": n * n * 4}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    bf16_peak, _, src = peaks()
    kern_tflops = flop / (kern_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "TFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": f"linalg.matmul precision sweep, BF16 in / FP32 accumulate, M=N=K={n}",
                   "inputs": "A, B ~ N(0,1) with 1% of entries x100 (SplitMix64 seed 3)",
                   "step": "cast A, cast+transpose B to BF16, tcgen05 GEMM (FP32 out)",
                   "l2": "inputs larger than L2 (268 MB FP32 per operand); no flush"},
        "roofline": {"bound": "tensor", "achieved": kern_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": kern_tflops / bf16_peak, "traffic": None,
                     "kernel": "tc_gemm_kernel<BF16,1>", "peak_source": f"{src} bf16 burst"},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        "e2e": e2e,
        "sweep": sweep,
        "accuracy": extra,
    }
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(A, B, args.cpu_rows)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
