"""GPU parity of the E4M3 convolution paths beyond the per-tap kernel.

* The stacked window kernel on E4M3 operands (schedule tile_k = 128 * KH:
  128-channel K blocks, tcgen05.mma kind::f8f6f4).  Half-integer inputs with
  amax 3.5 quantise to exact E4M3 codes under the scale 448 / 3.5 = 128, and
  every partial sum of their products is a multiple of 4096 below 2^24 * 4096,
  so the result must equal the FP64 oracle bit for bit.
* Operands the caller quantised once (nk_conv2d_pack_weights_fp8 for W, an
  amax and a cast for I) with their scales passed to the call: the same codes
  and the same dequantisation 1/(s_i s_w) as the per-call quantisation, so
  the two results are bitwise equal.
* The layers the E4M3 window kernel is for (C >= 128) at their tolerances:
  within 6e-2 of the FP32 convolution, within 1e-5 of the exact convolution
  of the dequantised operands.
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


def _half_ints(seed, stream, shape, edge):
    x = synth.small_ints(seed, stream, shape) / 2
    x.flat[0] = edge
    return x


CASES = [
    # N, H, W, C, F, KH, KW, dilation, pad (stride 1)
    (1, 9, 9, 128, 64, 3, 3, (1, 1), (1, 1, 1, 1)),
    (2, 13, 11, 200, 24, 3, 3, (1, 2), (1, 0, 2, 1)),    # two channel blocks, the second ragged
    (2, 10, 12, 256, 96, 3, 3, (1, 1), (1, 1, 1, 1)),    # two N tiles, weights streamed
    (1, 17, 19, 136, 48, 4, 4, (1, 1), (1, 2, 1, 2)),    # KW = 4: N = 256
    (3, 9, 11, 128, 40, 3, 2, (2, 1), (2, 2, 1, 1)),     # KW = 2, row dilation
    (5, 7, 7, 256, 72, 3, 3, (1, 1), (1, 1, 1, 1)),      # whole-width tiles: 7 wide at pitch 8
]


def _try_conv(nk, I, W, out, dl, pad, sched, **kw):
    try:
        nk.nk_conv2d_nhwc_hwcf(I, W, out, dilation=dl, pad=pad, precision="fp8", schedule=sched, **kw)
    except nk.NkError as e:
        if e.status == -7:   # no room for this schedule's layout on this shape
            pytest.skip(str(e))
        raise
    nk.nk_sync_status()
    return out


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("tm,stages", [(128, 1), (128, 2), (256, 4)])
def test_fp8_stacked_window_exact_codes_bitwise(nk, case, tm, stages):
    N, H, Wd, C, F, KH, KW, dl, pad = case
    I = _half_ints(111, H * 100 + C, (N, H, Wd, C), 3.5)
    W = _half_ints(112, F * 100 + KW, (KH, KW, C, F), -3.5)
    OH = O.conv_out_size(H, KH, 1, dl[0], pad[0], pad[1])
    OW = O.conv_out_size(Wd, KW, 1, dl[1], pad[2], pad[3])
    out = torch.full((N, OH, OW, F), float("nan"), device=DEV)
    _try_conv(nk, dev(I), dev(W), out, dl, pad, (tm, 64, 128 * KH, 1, stages, 1))
    np.testing.assert_array_equal(host(out), O.conv2d_nhwc_hwcf(I, W, (1, 1), dl, pad))


@pytest.mark.parametrize("sched", [None, (128, 128, 128, 1, 3, 1), (128, 64, 384, 1, 2, 1), (256, 64, 384, 1, 3, 1)])
def test_prequantised_operands_equal_per_call_quantisation(nk, sched):
    """Weights packed to E4M3 once and an input quantised once, scales given
    to the call: bitwise the result of the per-call quantisation."""
    N, H, Wd, C, F = 2, 14, 14, 128, 64
    I = synth.half_normal(113, 0, (N, H, Wd, C))
    W = synth.normal(113, 1, (3, 3, C, F), sigma=0.04)
    bias = synth.uniform(113, 2, (F,), -0.1, 0.1)
    i32, w32, b = dev(I), dev(W), dev(bias)
    ref = torch.empty(N, H, Wd, F, device=DEV)
    nk.nk_conv2d_nhwc_hwcf(i32, w32, ref, pad=(1, 1, 1, 1), precision="fp8", schedule=sched, bias=b, relu=True)
    wq, sw = nk.nk_conv2d_pack_weights_fp8(w32)
    iq, si = nk.quantize_nhwc_fp8(i32)
    got = torch.empty_like(ref)
    nk.nk_conv2d_nhwc_hwcf(iq, wq, got, pad=(1, 1, 1, 1), precision="fp8", schedule=sched, bias=b, relu=True,
                           scale_i=float(si.item()), scale_w=float(sw.item()))
    nk.nk_sync_status()
    np.testing.assert_array_equal(host(got), host(ref))
    # the scales are those of the format definition
    assert float(si.item()) == float(O.fp8_scale(I)) and float(sw.item()) == float(O.fp8_scale(W))


@pytest.mark.parametrize("shape", [(8, 28, 128, 128), (32, 14, 256, 256)])
def test_fp8_window_resnet_layers_within_tolerance(nk, shape):
    N, H, C, F = shape
    I, W, bias = synth.conv_resnet_block(N=N, H=H, W=H, C=C, F=F)
    i32, w32, b = dev(I), dev(W), dev(bias)
    wq, sw = nk.nk_conv2d_pack_weights_fp8(w32)
    iq, si = nk.quantize_nhwc_fp8(i32)
    out = torch.empty(N, H, H, F, device=DEV)
    nk.nk_conv2d_nhwc_hwcf(iq, wq, out, pad=(1, 1, 1, 1), precision="fp8", bias=b, relu=True,
                           scale_i=float(si.item()), scale_w=float(sw.item()))
    nk.nk_sync_status()
    got = host(out)
    R32 = O.epilogue(O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)), bias=bias, relu=True)
    assert O.rel_frobenius(got, R32) <= 6e-2
    s_i, s_w = O.fp8_scale(I), O.fp8_scale(W)
    Rq = O.conv2d_nhwc_hwcf(O.fp8_quantize(I, s_i), O.fp8_quantize(W, s_w), pad=(1, 1, 1, 1))
    Rq = O.epilogue(Rq / (np.float64(s_i) * np.float64(s_w)), bias=bias, relu=True)
    assert O.rel_frobenius(got, Rq) <= 1e-5


def test_fp8_default_uses_the_window_kernel_from_128_channels(nk):
    import paper_2307_16080_gb300.nk_tune as nt
    assert nt.nk_default_schedule(nt.conv_problem(8, 28, 28, 128, 128, 3, 3, 1, 1, "fp8"))[2] == 384
    assert nt.nk_default_schedule(nt.conv_problem(8, 56, 56, 64, 64, 3, 3, 1, 1, "fp8"))[2] == 128


def test_fp8_operand_combinations_rejected(nk):
    I = synth.half_normal(114, 0, (1, 8, 8, 128))
    W = synth.normal(114, 1, (3, 3, 128, 64), sigma=0.05)
    out = torch.empty(1, 8, 8, 64, device=DEV)
    wq, sw = nk.nk_conv2d_pack_weights_fp8(dev(W))
    iq, si = nk.quantize_nhwc_fp8(dev(I))
    for a, b, kw in [(dev(I), wq, {}),                                  # FP32 I with E4M3 W
                     (iq, dev(W), {}),                                  # E4M3 I with FP32 W
                     (iq, wq, {"scale_i": 0.0, "scale_w": 1.0}),        # no valid scale
                     (iq, nk.nk_conv2d_pack_weights(dev(W)), {})]:      # E4M3 I with BF16 W
        with pytest.raises(nk.NkError):
            nk.nk_conv2d_nhwc_hwcf(a, b, out, pad=(1, 1, 1, 1), precision="fp8", **kw)
    with pytest.raises(nk.NkError):   # E4M3 operands need the FP8 precision
        nk.nk_conv2d_nhwc_hwcf(iq, wq, out, pad=(1, 1, 1, 1), precision="bf16")
