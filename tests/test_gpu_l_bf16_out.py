"""GPU parity of convolutions that write BF16 outputs.

The epilogue computes in FP32 exactly as for an FP32 output (bias, ReLU,
accumulate, fused program) and rounds each result to BF16 with
round-to-nearest-even as it stores it.  On small-integer inputs every
product and partial sum is exact in FP32, so the stored value must equal the
oracle's bf16_rn of the exact FP64 result, bit for bit, on every kernel that
can write the output: the per-tap implicit GEMM (with and without split-K,
whose reduce then writes BF16), the shared-window kernel, the stacked
kernel-row kernel with one and with two accumulator buffers, and the E4M3
per-tap kernel.  With real-valued inputs the BF16 result is within half a
BF16 ulp of the FP32 result: |bf16_rn(x) - x| <= 2^-9 |x| per element.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import DEV, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


def _bf16_host(t):
    return t.float().cpu().numpy()


def _out(N, OH, OW, F, dtype=torch.bfloat16):
    return torch.full((N, OH, OW, F), float("nan"), device=DEV, dtype=dtype)


SCHEDS = [
    ("per-tap", (128, 64, 64, 1, 3, 1)),
    ("per-tap split-K", (128, 64, 64, 1, 3, 3)),
    ("per-tap pair", (256, 128, 64, 2, 4, 1)),
    ("window", (128, 64, 576, 1, 2, 1)),
    ("stacked", (128, 64, 192, 1, 1, 1)),
    ("stacked two buffers", (256, 64, 192, 1, 4, 1)),
]


@pytest.mark.parametrize("name,sched", SCHEDS)
@pytest.mark.parametrize("F", [64, 40, 12])   # F % 8 != 0: the scalar store path
def test_bf16_output_small_ints_bitwise(nk, name, sched, F):
    N, H, Wd, C = 2, 13, 15, 64
    I = synth.small_ints(101, F, (N, H, Wd, C))
    W = synth.small_ints(102, F, (3, 3, C, F))
    bias = synth.small_ints(103, F, (F,))
    out = _out(N, H, Wd, F)
    nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), out, pad=(1, 1, 1, 1), precision="bf16", schedule=sched,
                           bias=dev(bias), relu=True)
    nk.nk_sync_status()
    R = O.epilogue(O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)), bias=bias, relu=True)
    np.testing.assert_array_equal(_bf16_host(out), O.bf16_rn(R))


@pytest.mark.parametrize("name,sched", SCHEDS)
def test_bf16_output_accumulate_and_program(nk, name, sched):
    """accumulate = 1 reads the BF16 output as C_in; a fused program (ADD of
    an FP32 tensor, then ReLU) runs on the FP32 value before the rounding."""
    N, H, Wd, C, F = 2, 11, 12, 64, 64
    I = synth.small_ints(104, 0, (N, H, Wd, C))
    W = synth.small_ints(104, 1, (3, 3, C, F))
    C0 = synth.small_ints(104, 2, (N, H, Wd, F), -40, 40)
    T = synth.small_ints(104, 3, (N, H, Wd, F), -100, 100)
    out = dev(C0).to(torch.bfloat16)
    t = dev(T)
    nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), out, pad=(1, 1, 1, 1), precision="bf16", schedule=sched,
                           accumulate=True, ew=[("add", t), ("relu",)])
    nk.nk_sync_status()
    R = O.conv2d_fused(I, W, "bf16", pad=(1, 1, 1, 1), o_in=C0, beta=1.0, ew=[("add", T), ("relu",)])
    np.testing.assert_array_equal(_bf16_host(out), O.bf16_rn(R))


def test_bf16_output_within_half_an_ulp_of_fp32(nk):
    """The ResNet block in BF16 with packed weights: the BF16 output is the
    FP32 output rounded once, so elementwise |bf16 - fp32| <= 2^-9 |fp32|,
    and within 2^-9 + 1e-5 (Frobenius) of the oracle."""
    I, W, bias = synth.conv_resnet_block(N=4)
    i16, wp, b = dev(I).to(torch.bfloat16), nk.nk_conv2d_pack_weights(dev(W)), dev(bias)
    o32 = torch.empty(4, 56, 56, 64, device=DEV)
    o16 = _out(4, 56, 56, 64)
    for o in (o32, o16):
        nk.nk_conv2d_nhwc_hwcf(i16, wp, o, pad=(1, 1, 1, 1), precision="bf16", bias=b, relu=True)
    nk.nk_sync_status()
    f32, f16 = host(o32), _bf16_host(o16)
    np.testing.assert_array_equal(f16, O.bf16_rn(f32))
    R = O.epilogue(O.conv2d_nhwc_hwcf(O.bf16_rn(I), O.bf16_rn(W), pad=(1, 1, 1, 1)), bias=bias, relu=True)
    assert O.rel_frobenius(f16, R) <= 2.0 ** -9 + 1e-5


def test_fp8_conv_bf16_output_exact_codes(nk):
    """E4M3 per-tap kernel, dequantised by 1/(s_i s_w) in FP32, then BF16."""
    N, H, Wd, C, F = 2, 9, 10, 128, 64
    I = synth.small_ints(105, 0, (N, H, Wd, C)) / 2
    W = synth.small_ints(105, 1, (3, 3, C, F)) / 2
    I.flat[0], W.flat[0] = 3.5, -3.5
    out = _out(N, H, Wd, F)
    nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), out, pad=(1, 1, 1, 1), precision="fp8")
    nk.nk_sync_status()
    np.testing.assert_array_equal(_bf16_host(out), O.bf16_rn(O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1))))


def test_fp32_conv_rejects_bf16_output(nk):
    I = synth.small_ints(106, 0, (1, 8, 8, 16))
    W = synth.small_ints(106, 1, (3, 3, 16, 16))
    with pytest.raises(nk.NkError):
        nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), _out(1, 8, 8, 16), pad=(1, 1, 1, 1), precision="f32")
