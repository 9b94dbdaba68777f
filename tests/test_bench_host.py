"""Host logic of bench.py (no GPU): the roofline arithmetic behind every
reported fraction, the traffic record's source check, and the reference
arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

import bench
from paper_2307_16080_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_layer_roofline_closed_form_32x56x56x64():
    """3x3, 64 -> 64, pad 1 at batch 32: 2*N*OH*OW*F*KH*KW*C FLOP; BF16 in
    (2 B), FP32 out (4 B), BF16 weights once."""
    r = bench.layer_roofline(32, 56, 56, 64, 64, 3, 3, 1, 1, ms=0.0174)
    assert r["flop"] == 2.0 * 32 * 56 * 56 * 64 * 9 * 64 == 7398752256.0
    assert r["bytes"] == 2.0 * 32 * 56 * 56 * 64 + 4.0 * 32 * 56 * 56 * 64 + 2.0 * 9 * 64 * 64 == 38608896.0
    peak, hbm, _ = bench.peaks()
    ai = r["flop"] / r["bytes"]
    assert r["ai_flop_per_byte"] == pytest.approx(ai)
    roof = min(peak, hbm * 1e-3 * ai)
    assert r["roofline_tflops"] == pytest.approx(roof)
    assert r["bound"] == ("hbm" if hbm * 1e-3 * ai < peak else "tensor")
    assert r["achieved_tflops"] == pytest.approx(7398752256.0 / 0.0174e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved_tflops"] / roof)


def test_layer_roofline_output_and_input_widths():
    """BF16 output halves the output bytes; E4M3 operands halve input and
    weight bytes; a large enough peak leaves the HBM bound in place."""
    a = bench.layer_roofline(8, 28, 28, 128, 128, 3, 3, 1, 1, 1.0, out_bytes=4, in_bytes=2)
    b = bench.layer_roofline(8, 28, 28, 128, 128, 3, 3, 1, 1, 1.0, out_bytes=2, in_bytes=2)
    c = bench.layer_roofline(8, 28, 28, 128, 128, 3, 3, 1, 1, 1.0, out_bytes=4, in_bytes=1, peak=1e9)
    n_in, n_out, n_w = 8 * 28 * 28 * 128, 8 * 28 * 28 * 128, 9 * 128 * 128
    assert a["bytes"] - b["bytes"] == 2.0 * n_out
    assert a["bytes"] - c["bytes"] == 1.0 * (n_in + n_w)
    assert c["bound"] == "hbm"


def test_stack_roofline_is_the_sum_of_layer_rooflines():
    for batch in (1, 32):
        want = 0.0
        for L in synth.resnet_stack(batch):
            r = bench.layer_roofline(L["N"], L["H"], L["W"], L["C"], L["F"], L["KH"], L["KW"], L["stride"],
                                     L["pad"], 1.0)
            want += r["flop"] / (r["roofline_tflops"] * 1e12) * 1e3
        assert bench.stack_roofline_ms(synth, batch) == pytest.approx(want)
        assert bench.stack_roofline_ms(synth, batch, [4] * 20) == pytest.approx(want)
        # BF16 outputs everywhere: fewer bytes, never a slower roofline
        assert bench.stack_roofline_ms(synth, batch, 2) <= want


def test_recorded_traffic_only_for_the_captured_source(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["tc_gemm_bf16_8192"]
    if rec["source_sha256"] == bench.source_sha():
        assert bench.recorded_traffic("tc_gemm_bf16_8192") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "source_sha", lambda: "0" * 64)
    assert bench.recorded_traffic("tc_gemm_bf16_8192") is None
    assert bench.recorded_traffic("no such kernel") is None


def test_reference_arm_prints_one_json_line():
    """--impl reference times the FP64 oracle on the host (no GPU): one
    JSON line with the contract's keys and zero host-device bytes."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-rows", "8"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "TFLOP/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
