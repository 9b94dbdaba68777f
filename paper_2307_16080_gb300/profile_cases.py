"""Fixed workloads for the library's kernels, one family at a time, timed with
CUDA events and reported against the measured peaks -- the commands the
ncu summaries under profiles/ were taken with.

  python -m paper_2307_16080_gb300.profile_cases CASE [--reps R]

CASE:
  cast      FP32 8192 x 8192 -> BF16, row-major and transposed (operand prep)
  amax      max |x| over 8192 x 8192 FP32
  direct    NCHW conv, Ci = 1, Co = 3, 3 x 3 on 1280 x 1280 images, batch 1
            (the tuning experiment's shape) and batch 16 (larger than L2)
  conv      BF16 conv, batch 32 x 56 x 56 x 64, 3 x 3 x 64 x 64, built-in schedule (the
            shared-window kernel)
  conv_tap  the same layer on the per-tap implicit-GEMM kernel, schedule (128, 64, 64, 1, 3, 1)
  grouped   512 uneven BF16 GEMMs, one persistent launch, tile chosen by nk_grouped_tune
  splitk    FP32 1024 x 1024 x 16384 with split-K 8 (partials + fixed-order reduce)
Prints one JSON line per measurement.  Times are device times: `calls`
back-to-back calls captured into a CUDA graph, replayed between CUDA events.
"""
from __future__ import annotations

import argparse
import json
import os

import torch

from . import nk, synth


def _peaks():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"])
    except Exception:
        return 6800.0, 1900.0


def _time(fn, reps, calls=4):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(calls):
                fn()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    nk.nk_sync_status()
    return e0.elapsed_time(e1) / (reps * calls)


def _emit(case, ms, bytes_=None, flop=None):
    hbm, bf16 = _peaks()
    out = {"case": case, "ms": ms}
    if bytes_ is not None:
        gbs = bytes_ / (ms * 1e-3) / 1e9
        out.update({"algorithmic_bytes": bytes_, "GB/s": gbs, "frac_of_measured_hbm": gbs / hbm})
    if flop is not None:
        tf = flop / (ms * 1e-3) / 1e12
        out.update({"flop": flop, "TFLOP/s": tf, "frac_of_measured_bf16": tf / bf16})
    print(json.dumps(out), flush=True)


def case_cast(reps):
    n = 8192
    x = torch.randn(n, n, device="cuda")
    y = torch.empty(n, n, dtype=torch.bfloat16, device="cuda")
    _emit("cast_rows bf16 8192^2", _time(lambda: nk.nk_cast_bf16(x, y), reps), bytes_=n * n * 6)
    _emit("cast_transpose bf16 8192^2", _time(lambda: nk.nk_cast_bf16(x, y, transpose=True), reps), bytes_=n * n * 6)


def case_amax(reps):
    n = 8192
    x = torch.randn(n, n, device="cuda")
    a = torch.empty(1, device="cuda")
    ws = nk.workspace(nk.lib().nk_prep_workspace_size(n * n))
    _emit("amax 8192^2", _time(lambda: nk.nk_amax(x, a, ws), reps), bytes_=n * n * 4)


def case_direct(reps):
    for batch in (1, 16):
        i = torch.randn(batch, 1, 1280, 1280, device="cuda")
        k = torch.randn(3, 1, 3, 3, device="cuda")
        o = torch.empty(batch, 3, 1278, 1278, device="cuda")
        b = batch * (1280 * 1280 + 3 * 1278 * 1278) * 4
        f = 2.0 * batch * 3 * 1278 * 1278 * 9
        _emit(f"direct nchw conv ({batch},1,1280,1280) Co=3 3x3",
              _time(lambda: nk.nk_conv2d_nchw_fchw(i, k, o), reps), bytes_=b, flop=f)


def _conv_layer(reps, sched, name):
    N, H, C, F = 32, 56, 64, 64
    i = torch.randn(N, H, H, C, device="cuda").abs().to(torch.bfloat16)
    w = torch.randn(3, 3, C, F, device="cuda") * 0.06
    o = torch.empty(N, H, H, F, device="cuda")
    ws = nk.workspace(nk.nk_conv2d_workspace_size(i, w, o, pad=(1, 1, 1, 1), precision="bf16", schedule=sched))
    f = 2.0 * N * H * H * F * 9 * C
    b = N * H * H * (C * 2 + F * 4) + 9 * C * F * 4   # BF16 input, FP32 output, FP32 weights
    _emit(name, _time(lambda: nk.nk_conv2d_nhwc_hwcf(i, w, o, pad=(1, 1, 1, 1), precision="bf16", schedule=sched,
                                                     ws=ws), reps), bytes_=b, flop=f)


def case_conv(reps):
    _conv_layer(reps, None, "bf16 conv 32x56x56x64 3x3 (built-in schedule)")


def case_conv_window(reps):
    _conv_layer(reps, (128, 64, 576, 1, 1, 1), "bf16 conv 32x56x56x64 3x3 (window kernel, taps in K)")


def case_conv_tap(reps):
    _conv_layer(reps, (128, 64, 64, 1, 3, 1), "bf16 conv 32x56x56x64 3x3 (per-tap kernel)")


def case_stack8(reps):
    """The 20-layer ResNet-style stack at batch 8: packed BF16 weights, BF16
    activations, built-in schedules, one nk_conv2d call per layer."""
    calls, flop = [], 0.0
    for L in synth.resnet_stack(8):
        oh = (L["H"] + 2 * L["pad"] - L["KH"]) // L["stride"] + 1
        x = torch.randn(L["N"], L["H"], L["W"], L["C"], device="cuda").abs().to(torch.bfloat16)
        w = nk.nk_conv2d_pack_weights(torch.randn(L["KH"], L["KW"], L["C"], L["F"], device="cuda") * 0.05)
        b = torch.randn(L["F"], device="cuda") * 0.1
        o = torch.empty(L["N"], oh, oh, L["F"], device="cuda")
        st, pd = (L["stride"],) * 2, (L["pad"],) * 4
        ws = nk.workspace(nk.nk_conv2d_workspace_size(x, w, o, st, (1, 1), pd, "bf16"))
        calls.append((x, w, o, st, pd, b, ws))
        flop += 2.0 * L["N"] * oh * oh * L["F"] * L["KH"] * L["KW"] * L["C"]

    def forward():
        for (x, w, o, st, pd, b, ws) in calls:
            nk.nk_conv2d_nhwc_hwcf(x, w, o, st, (1, 1), pd, "bf16", bias=b, relu=True, ws=ws)
    _emit("resnet stack batch 8, 20 convs (built-in schedules)", _time(forward, reps), flop=flop)


def case_grouped(reps):
    shapes = [tuple(int(v) for v in s) for s in synth.grouped_problems(512)]
    a = [torch.empty(M, K, device="cuda").uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in shapes]
    bt = [torch.empty(N, K, device="cuda").uniform_(-1, 1).to(torch.bfloat16) for (M, N, K) in shapes]
    c = [torch.empty(M, N, device="cuda") for (M, N, K) in shapes]
    groups, G = nk.make_groups(a, bt, c)
    from . import nk_tune as nt
    best, _ = nt.nk_grouped_tune(groups, G, reps=3)
    plan = nk.nk_grouped_plan_create(groups, G, schedule=best)
    f = float(sum(2.0 * M * N * K for (M, N, K) in shapes))
    _emit("grouped 512 bf16 gemms", _time(lambda: nk.nk_grouped_plan_run(plan), reps), flop=f)
    nk.nk_grouped_plan_destroy(plan)


def case_splitk(reps):
    M, N, K, s = 1024, 1024, 16384, 8
    a = torch.randn(M, K, device="cuda")
    b = torch.randn(K, N, device="cuda")
    c = torch.empty(M, N, device="cuda")
    sched = (64, 64, 16, 1, 2, s)
    ws = nk.workspace(nk.nk_matmul_workspace_size(a, b, c, "f32", sched))
    _emit("f32 split-K 8 1024x1024x16384", _time(
        lambda: nk.nk_matmul(a, b, c, precision="f32", schedule=sched, ws=ws), reps), flop=2.0 * M * N * K)


CASES = {"cast": case_cast, "amax": case_amax, "direct": case_direct, "conv": case_conv, "conv_window": case_conv_window, "stack8": case_stack8,
         "conv_tap": case_conv_tap,
         "grouped": case_grouped, "splitk": case_splitk}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args()
    nk.lib()
    CASES[a.case](a.reps)


if __name__ == "__main__":
    main()
