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
