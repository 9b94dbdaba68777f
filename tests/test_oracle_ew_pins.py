"""Pins for the oracle's fused elementwise programs (CPU only).

The activations are tied to closed forms and to torch's independent FP64 CPU
routines; program order, operand placement and the prologue's interplay with
padding and quantisation are tied to hand-computed results and to exact
invariants of power-of-two scaling.
"""
import math

import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth

X = np.linspace(-8.0, 8.0, 2001)


def _torch(fn, x):
    return fn(torch.from_numpy(np.asarray(x, np.float64))).numpy()


def test_sigmoid_silu_tanh_closed_forms():
    ln3, ln2 = math.log(3.0), math.log(2.0)
    # sigma(ln 3) = 1 / (1 + 1/3) = 3/4; silu(ln 3) = (3/4) ln 3; tanh(ln 2) = (2 - 1/2) / (2 + 1/2) = 3/5
    assert abs(O.sigmoid(np.array([ln3]))[0] - 0.75) < 1e-15
    assert abs(O.silu(np.array([ln3]))[0] - 0.75 * ln3) < 1e-15
    assert abs(O.ew_program(np.array([ln2]), [("tanh",)])[0] - 0.6) < 1e-15
    assert O.sigmoid(np.array([0.0]))[0] == 0.5
    np.testing.assert_allclose(O.sigmoid(X) + O.sigmoid(-X), 1.0, atol=1e-15)
    np.testing.assert_allclose(O.silu(X) - O.silu(-X), X, atol=1e-14)
    # tanh(x) = 2 sigma(2x) - 1 ties the tanh step to the logistic function
    np.testing.assert_allclose(O.ew_program(X, [("tanh",)]), 2 * O.sigmoid(2 * X) - 1, atol=1e-15)
    # no overflow at the ends
    s = O.sigmoid(np.array([-1000.0, 1000.0]))
    assert s[0] == 0.0 and s[1] == 1.0


def test_activations_match_torch_fp64():
    np.testing.assert_allclose(O.sigmoid(X), _torch(torch.sigmoid, X), rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(O.silu(X), _torch(torch.nn.functional.silu, X), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(O.gelu_tanh(X), _torch(lambda t: torch.nn.functional.gelu(t, approximate="tanh"), X),
                               rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(O.ew_program(X, [("gelu",)]), _torch(torch.nn.functional.gelu, X),
                               rtol=1e-14, atol=1e-15)


def test_gelu_tanh_is_close_to_exact_gelu():
    # the approximation stays within 1e-3 of x*Phi(x); a dropped cubic term is off by ~3e-2
    assert np.max(np.abs(O.gelu_tanh(X) - O.gelu(X))) < 1e-3
    assert O.gelu_tanh(np.array([0.0]))[0] == 0.0
    assert abs(O.gelu_tanh(np.array([10.0]))[0] - 10.0) < 1e-12


def test_program_order_and_tensor_operands_by_hand():
    x = np.array([3.0, -1.0])
    T = np.array([5.0, 2.0])
    # (2x + 1) * T = [35, -2]; 2 (x T) + 1 = [31, -3]
    np.testing.assert_array_equal(O.ew_program(x, [("affine", 2, 1), ("mul", T)]), [35.0, -2.0])
    np.testing.assert_array_equal(O.ew_program(x, [("mul", T), ("affine", 2, 1)]), [31.0, -3.0])
    # add then relu vs relu then add
    np.testing.assert_array_equal(O.ew_program(x, [("add", T), ("relu",)]), [8.0, 1.0])
    np.testing.assert_array_equal(O.ew_program(np.array([-3.0]), [("relu",), ("add", np.array([-2.0]))]), [-2.0])
    out = O.ew_program(np.array([-3.0, 0.5, 5.0, np.nan]), [("clamp", -1, 1)])
    np.testing.assert_array_equal(out[:3], [-1.0, 0.5, 1.0])
    assert np.isnan(out[3])
    assert np.isnan(O.ew_program(np.array([np.nan]), [("relu",)])[0])
    np.testing.assert_array_equal(O.ew_program(x, None), x)
    with pytest.raises(ValueError):
        O.ew_program(x, [("exp",)])


def test_matmul_fused_places_prologues_and_epilogue_by_hand():
    A = np.array([[1.0, -2.0], [3.0, 4.0]], np.float32)
    B = np.array([[-1.0, 2.0], [3.0, -4.0]], np.float32)
    eye = np.eye(2, dtype=np.float32)
    # relu(A) @ I
    np.testing.assert_array_equal(O.matmul_fused(A, eye, pro_a=[("relu",)]), [[1.0, 0.0], [3.0, 4.0]])
    # I @ relu(B)
    np.testing.assert_array_equal(O.matmul_fused(eye, B, pro_b=[("relu",)]), [[0.0, 2.0], [3.0, 0.0]])
    # epilogue order: bias, ReLU, then the program:  relu(A@I + [1, 1]) * T
    T = np.array([[2.0, 3.0], [4.0, 5.0]])
    got = O.matmul_fused(A, eye, bias=np.array([1.0, 1.0]), relu=True, ew=[("mul", T)])
    np.testing.assert_array_equal(got, [[4.0, 0.0], [16.0, 25.0]])
    # accumulate: beta*C_in enters before the program
    got = O.matmul_fused(A, eye, c_in=np.ones((2, 2)), beta=1.0, ew=[("affine", 10, 0)])
    np.testing.assert_array_equal(got, [[20.0, -10.0], [40.0, 50.0]])


def test_matmul_fused_equals_loops_on_small_ints():
    A = synth.uniform(60, 0, (5, 7))
    B = synth.uniform(60, 1, (7, 3))
    A = np.round(A * 4).astype(np.float32)
    B = np.round(B * 4).astype(np.float32)
    T = np.round(synth.uniform(60, 2, (5, 3)) * 4)
    want = O.matmul_loops(np.maximum(A, 0), B * 2.0) + T
    got = O.matmul_fused(A, B, pro_a=[("relu",)], pro_b=[("affine", 2, 0)], ew=[("add", T)])
    np.testing.assert_array_equal(got, want)


def test_conv_prologue_leaves_padding_zero():
    # every input value becomes 1 (0*x + 1); W sums a 3x3 window of one channel.
    # Zero padding stays zero, so corners see 4 ones, edges 6, the interior 9.
    I = synth.normal(61, 0, (1, 4, 5, 1))
    W = np.ones((3, 3, 1, 1), np.float32)
    O_ = O.conv2d_fused(I, W, pad=(1, 1, 1, 1), pro_i=[("affine", 0, 1)])[0, :, :, 0]
    want = np.array([[4, 6, 6, 6, 4], [6, 9, 9, 9, 6], [6, 9, 9, 9, 6], [4, 6, 6, 6, 4]], np.float64)
    np.testing.assert_array_equal(O_, want)


@pytest.mark.parametrize("precision", ["bf16", "fp8", "bf16x3"])
def test_power_of_two_prologue_commutes_with_quantisation(precision):
    # Scaling an operand by 1/2 before the conversion halves the result exactly:
    # BF16 / BF16x3 rounding commutes with powers of two, and for E4M3 the
    # per-tensor scale (taken from the transformed operand) absorbs the factor.
    A, B = synth.matmul_outlier(24, 40, 32, seed=62)
    base = O.matmul_fused(A, B, precision)
    half = O.matmul_fused(A, B, precision, pro_a=[("affine", 0.5, 0)])
    np.testing.assert_array_equal(half, 0.5 * base)
    I = synth.normal(63, 0, (2, 6, 6, 8))
    W = synth.normal(63, 1, (3, 3, 8, 4))
    if precision != "bf16x3":
        cb = O.conv2d_fused(I, W, precision, pad=(1, 1, 1, 1))
        ch = O.conv2d_fused(I, W, precision, pad=(1, 1, 1, 1), pro_w=[("affine", 0.5, 0)])
        np.testing.assert_array_equal(ch, 0.5 * cb)


def test_prologue_rounds_to_fp32_once():
    x = np.array([1.0 + 2.0 ** -30], np.float64)
    out = O.prologue(x, [("affine", 1.0, 0.0)])
    assert out.dtype == np.float32 and out[0] == np.float32(1.0)
