"""GPU parity of the window convolution with stacked kernel rows.

Schedule tile_k = 64 * KH selects it: for each kernel row the KW taps sit
side by side along the MMA's N (N = 64 * KW), and the epilogue adds each
tap's partial sums from the rows kw * dw further on.  Small-integer inputs
make every product and partial sum exact, so the result must equal the
FP64 oracle bit for bit, whatever the order of the additions.
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


def _conv(nk, I, W, dl, pad, sched, **kw):
    N, H, Wd, C = I.shape
    KH, KW, _, F = W.shape
    OH = O.conv_out_size(H, KH, 1, dl[0], pad[0], pad[1])
    OW = O.conv_out_size(Wd, KW, 1, dl[1], pad[2], pad[3])
    out = kw.pop("out", None)
    if out is None:
        out = torch.full((N, OH, OW, F), float("nan"), device=DEV)
    i = kw.pop("i_dev", None)
    w = kw.pop("w_dev", None)
    nk.nk_conv2d_nhwc_hwcf(dev(I) if i is None else i, dev(W) if w is None else w, out, dilation=dl, pad=pad,
                           precision="bf16", schedule=sched, **kw)
    nk.nk_sync_status()
    return host(out)


STACK_CASES = [
    # N, H, W, C, F, KH, KW, dilation, pad  (stride 1)
    (1, 8, 8, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),
    (2, 13, 11, 16, 24, 3, 3, (1, 2), (1, 0, 2, 1)),     # column dilation, F < 64
    (1, 12, 12, 5, 7, 3, 3, (1, 1), (0, 0, 0, 0)),       # C not a multiple of 8
    (2, 9, 9, 200, 72, 3, 3, (1, 1), (1, 1, 1, 1)),      # 4 channel blocks, 2 N tiles, weights streamed
    (1, 20, 18, 32, 130, 3, 2, (2, 1), (2, 2, 1, 1)),    # KW = 2, row dilation, 3 N tiles
    (3, 9, 11, 40, 96, 3, 3, (1, 1), (1, 1, 1, 1)),      # several images per window (P = 8)
    (1, 6, 140, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),     # rows wider than one window
    (2, 17, 19, 64, 48, 4, 4, (1, 1), (1, 2, 1, 2)),     # KW = 4: N = 256
    (2, 17, 19, 64, 48, 2, 2, (1, 1), (0, 1, 0, 1)),
    (2, 21, 23, 64, 64, 3, 3, (2, 2), (2, 2, 2, 2)),     # P = 32
    (2, 15, 17, 96, 160, 3, 3, (1, 1), (1, 1, 1, 1)),
    # whole-width tiles (one column tile, shifts past the window row read
    # right padding and are left out): 7 and 15 wide, asymmetric pads, dilation
    (4, 7, 7, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),
    (3, 7, 7, 96, 130, 3, 3, (1, 1), (1, 1, 0, 2)),
    (2, 15, 15, 64, 48, 3, 3, (1, 1), (1, 1, 1, 1)),
    (2, 13, 13, 64, 64, 3, 3, (2, 2), (2, 2, 2, 2)),
]


@pytest.mark.parametrize("case", STACK_CASES)
@pytest.mark.parametrize("stages", [1, 2, 4])
def test_bf16_conv_stacked_bitwise(nk, case, stages):
    N, H, Wd, C, F, KH, KW, dl, pad = case
    I = synth.small_ints(91, H * 100 + C, (N, H, Wd, C))
    W = synth.small_ints(91, F * 100 + KH * 10 + KW, (KH, KW, C, F))
    got = _conv(nk, I, W, dl, pad, (128, 64, 64 * KH, 1, stages, 1))
    np.testing.assert_array_equal(got, O.conv2d_nhwc_hwcf(I, W, (1, 1), dl, pad))


def _legal(nk, case, sched):
    from paper_2307_16080_gb300 import nk_tune as nt
    N, H, Wd, C, F, KH, KW, dl, pad = case
    try:
        nt.nk_conv_window_tile(N, H, Wd, C, F, KH, KW, dl, pad, sched)
        return True
    except nk.NkError:
        return False


@pytest.mark.parametrize("case", STACK_CASES)
@pytest.mark.parametrize("stages", [2, 5, 8])
def test_bf16_conv_stacked_double_buffered_bitwise(nk, case, stages):
    """tile_m 256: the same stacked tiles with two accumulator buffers and a
    deeper window ring (one CTA per SM); bit-exact on small integers."""
    N, H, Wd, C, F, KH, KW, dl, pad = case
    sched = (256, 64, 64 * KH, 1, stages, 1)
    if not _legal(nk, case, sched):
        pytest.skip("no room for this many window slots beside the filters")
    I = synth.small_ints(91, H * 100 + C, (N, H, Wd, C))
    W = synth.small_ints(91, F * 100 + KH * 10 + KW, (KH, KW, C, F))
    got = _conv(nk, I, W, dl, pad, sched)
    np.testing.assert_array_equal(got, O.conv2d_nhwc_hwcf(I, W, (1, 1), dl, pad))


def test_double_buffered_schedules_exist_for_the_resnet_layers(nk):
    """Every stride-1 3x3 layer of the stack has at least one legal
    double-buffered stacked schedule with two or more window slots."""
    for L in synth.resnet_stack(8):
        if L["stride"] != 1 or L["KH"] != 3:
            continue
        case = (L["N"], L["H"], L["W"], L["C"], L["F"], 3, 3, (1, 1), (1, 1, 1, 1))
        assert any(_legal(nk, case, (256, 64, 192, 1, st, 1)) for st in range(2, 9)), L


@pytest.mark.parametrize("N", [1, 8, 32])
@pytest.mark.parametrize("tile_m,stages", [(256, 4)])
def test_bf16_conv_stacked_double_buffered_resnet_layer(nk, N, tile_m, stages):
    I, W, bias = synth.conv_resnet_block(N=N)
    i16, wp, b = dev(I).to(torch.bfloat16), nk.nk_conv2d_pack_weights(dev(W)), dev(bias)
    got = _conv(nk, I, W, (1, 1), (1, 1, 1, 1), (tile_m, 64, 192, 1, stages, 1), i_dev=i16, w_dev=wp, bias=b,
                relu=True)
    plain = _conv(nk, I, W, (1, 1), (1, 1, 1, 1), (128, 64, 576, 1, 1, 1), i_dev=i16, w_dev=wp, bias=b, relu=True)
    assert O.rel_frobenius(got, plain) <= 1e-5


@pytest.mark.parametrize("N", [1, 8, 32])
def test_bf16_conv_stacked_resnet_layer(nk, N):
    """The 56x56x64 3x3 layer of the ResNet-style stack, packed weights,
    bias + ReLU: within 1e-5 of the plain window kernel (only the order of
    additions differs) and, at batch 1 and 8, of the oracle on the
    bf16-rounded operands."""
    I, W, bias = synth.conv_resnet_block(N=N)
    i16, wp, b = dev(I).to(torch.bfloat16), nk.nk_conv2d_pack_weights(dev(W)), dev(bias)
    got = _conv(nk, I, W, (1, 1), (1, 1, 1, 1), (128, 64, 192, 1, 1, 1), i_dev=i16, w_dev=wp, bias=b, relu=True)
    plain = _conv(nk, I, W, (1, 1), (1, 1, 1, 1), (128, 64, 576, 1, 1, 1), i_dev=i16, w_dev=wp, bias=b, relu=True)
    assert O.rel_frobenius(got, plain) <= 1e-5
    if N <= 8:
        R = O.epilogue(O.conv2d_nhwc_hwcf(O.bf16_rn(I), O.bf16_rn(W), pad=(1, 1, 1, 1)), bias=bias, relu=True)
        assert O.rel_frobenius(got, R) <= 1e-5


def test_bf16_conv_stacked_epilogue_and_program(nk):
    """Bias, ReLU, accumulate and a fused program whose operand is the
    output itself (read before the store) through the stacked kernel."""
    N, H, Wd, C, F = 3, 19, 23, 64, 96
    I = synth.normal(92, 0, (N, H, Wd, C))
    W = synth.normal(92, 1, (3, 3, C, F), sigma=0.06)
    bias = synth.uniform(92, 2, (F,), lo=-0.1, hi=0.1)
    C0 = synth.uniform(92, 3, (N, H, Wd, F))
    out = dev(C0)
    got = _conv(nk, I, W, (1, 1), (1, 1, 1, 1), (128, 64, 192, 1, 2, 1), i_dev=dev(I).to(torch.bfloat16),
                out=out, bias=dev(bias), relu=True, accumulate=True, ew=[("add", out), ("gelu",)])
    R = O.conv2d_fused(I, W, "bf16", pad=(1, 1, 1, 1), o_in=C0, bias=bias, relu=True, beta=1.0,
                       ew=[("add", C0), ("gelu",)])
    assert O.rel_frobenius(got, R) <= 1e-5


@pytest.mark.parametrize("sched,stride,k", [
    ((128, 128, 192, 1, 1, 1), 1, 3),    # stacked N is 64 filters per tile
    ((512, 64, 192, 1, 2, 1), 1, 3),     # one chain, at most two accumulator buffers
    ((256, 64, 192, 1, 9, 1), 1, 3),     # at most 8 window slots
    ((128, 64, 192, 1, 1, 1), 2, 3),     # stride 1 only
    ((128, 64, 320, 1, 1, 1), 1, 5),     # KW = 5 would need N = 320
])
def test_bf16_conv_stacked_rejections(nk, sched, stride, k):
    I = synth.small_ints(93, 0, (1, 12, 12, 64))
    W = synth.small_ints(93, 1, (k, k, 64, 64))
    OH = O.conv_out_size(12, k, stride, 1, k // 2, k // 2)
    out = torch.empty(1, OH, OH, 64, device=DEV)
    with pytest.raises(nk.NkError):
        nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), out, stride=(stride, stride), pad=(k // 2,) * 4,
                               precision="bf16", schedule=sched)
