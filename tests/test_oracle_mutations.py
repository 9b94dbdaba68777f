"""Plant plausible mistakes in the oracle (on the CPU) and check a pin catches each.

Every mutant below is a one-line slip -- a flipped kernel, truncation in place
of round-to-nearest-even, a dropped term -- applied with monkeypatch to the
oracle only; the pins it must trip are re-run against the mutant.
"""
import numpy as np
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth


def test_flipped_conv_kernel_is_caught(monkeypatch):
    orig = O.conv2d_nhwc_hwcf
    monkeypatch.setattr(O, "conv2d_nhwc_hwcf",
                        lambda I, W, *a, **k: orig(I, np.asarray(W)[::-1, ::-1], *a, **k))
    I = synth.normal(50, 0, (1, 6, 6, 2))
    W = synth.normal(50, 1, (3, 3, 2, 2))
    assert O.rel_frobenius(O.conv2d_nhwc_hwcf(I, W), O.conv2d_loops(I, W)) > 1e-3


def test_truncating_bf16_is_caught(monkeypatch):
    def trunc(x):
        x = np.asarray(x, np.float32)
        return (x.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    monkeypatch.setattr(O, "bf16_rn", trunc)
    x = synth.normal(51, 0, (4096,))
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.any(O.bf16_rn(x) != want)


def test_dropped_cross_term_in_bf16x3_is_caught(monkeypatch):
    def bad(A32, B32, precision):
        (ah, al), (bh, bl) = O.prepared_operands(A32, B32, "bf16x3")[0]
        return O.matmul(ah, bh) + O.matmul(ah, bl)
    A, B = synth.matmul_outlier(64, 64, 256, seed=52)
    R = O.matmul(A, B)
    assert O.rel_frobenius(bad(A, B, "bf16x3"), R) > 2e-5
    assert O.rel_frobenius(O.matmul_precision(A, B, "bf16x3"), R) < 2e-5


def test_wrong_gelu_grad_sign_is_caught():
    x = np.linspace(-3, 3, 61)
    h = 1e-6
    fd = (O.gelu(x + h) - O.gelu(x - h)) / (2 * h)
    from scipy.special import erf
    Phi = 0.5 * (1 + erf(x / np.sqrt(2)))
    bad = Phi - x * np.exp(-0.5 * x * x) / np.sqrt(2 * np.pi)
    assert np.max(np.abs(bad - fd)) > 1e-2
    assert np.max(np.abs(O.gelu_grad(x) - fd)) < 1e-8


# ------------------------------------------------------------ elementwise programs
def test_dropped_cubic_term_in_gelu_tanh_is_caught():
    x = np.linspace(-8, 8, 2001)
    bad = 0.5 * x * (1 + np.tanh(np.sqrt(2 / np.pi) * x))
    assert np.max(np.abs(bad - O.gelu(x))) > 1e-2
    assert np.max(np.abs(O.gelu_tanh(x) - O.gelu(x))) < 1e-3


def test_reversed_program_order_is_caught(monkeypatch):
    orig = O.ew_program
    monkeypatch.setattr(O, "ew_program", lambda x, prog: orig(x, list(prog or ())[::-1]))
    x, T = np.array([3.0, -1.0]), np.array([5.0, 2.0])
    assert not np.array_equal(O.ew_program(x, [("affine", 2, 1), ("mul", T)]), [35.0, -2.0])


def test_prologue_on_the_wrong_operand_is_caught(monkeypatch):
    orig = O.matmul_fused
    monkeypatch.setattr(O, "matmul_fused",
                        lambda A, B, precision="f32", pro_a=None, pro_b=None, **k: orig(A, B, precision, pro_b, pro_a, **k))
    A = np.array([[1.0, -2.0], [3.0, 4.0]], np.float32)
    got = O.matmul_fused(A, np.eye(2, dtype=np.float32), pro_a=[("relu",)])
    assert not np.array_equal(got, [[1.0, 0.0], [3.0, 4.0]])


def test_prologue_applied_to_the_padding_is_caught():
    # the slip: pad first, then transform (the padding becomes 1, not 0)
    I = synth.normal(61, 0, (1, 4, 5, 1))
    W = np.ones((3, 3, 1, 1), np.float32)
    Ip = np.pad(np.asarray(I, np.float64), ((0, 0), (1, 1), (1, 1), (0, 0)))
    bad = O.conv2d_nhwc_hwcf(O.ew_program(Ip, [("affine", 0, 1)]), W)[0, :, :, 0]
    assert bad[0, 0] == 9.0   # the pin expects 4 at a corner
    good = O.conv2d_fused(I, W, pad=(1, 1, 1, 1), pro_i=[("affine", 0, 1)])[0, :, :, 0]
    assert good[0, 0] == 4.0


def test_fp8_scale_taken_before_the_prologue_is_caught():
    # the slip: s from amax(A) instead of amax(prologue(A))
    A, B = synth.matmul_outlier(24, 40, 32, seed=62)
    Ah = O.prologue(A, [("affine", 0.5, 0)])
    sa_wrong, sb = O.fp8_scale(A), O.fp8_scale(B)
    bad = O.matmul(O.fp8_quantize(Ah, sa_wrong), O.fp8_quantize(B, sb)) / (float(sa_wrong) * float(sb))
    base = O.matmul_fused(A, B, "fp8")
    assert not np.array_equal(bad, 0.5 * base)
    np.testing.assert_array_equal(O.matmul_fused(A, B, "fp8", pro_a=[("affine", 0.5, 0)]), 0.5 * base)
