"""GPU parity of the BF16 tensor-core implicit-GEMM convolution
(linalg.conv_2d_nhwc_hwcf) against the FP64 oracle, through the C ABI."""
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


def _conv(nk, I, W, st, dl, pad, **kw):
    N, H, Wd, C = I.shape
    KH, KW, _, F = W.shape
    OH = O.conv_out_size(H, KH, st[0], dl[0], pad[0], pad[1])
    OW = O.conv_out_size(Wd, KW, st[1], dl[1], pad[2], pad[3])
    out = torch.empty(N, OH, OW, F, device=DEV)
    i = kw.pop("i_dev", None)
    nk.nk_conv2d_nhwc_hwcf(dev(I) if i is None else i, dev(W), out, stride=st, dilation=dl, pad=pad,
                           precision="bf16", **kw)
    nk.nk_sync_status()
    return host(out)


def test_bf16_conv_resnet_block(nk):
    I, W, bias = synth.conv_resnet_block()
    got = _conv(nk, I, W, (1, 1), (1, 1), (1, 1, 1, 1), bias=dev(bias), relu=True)
    R16 = O.epilogue(O.conv2d_nhwc_hwcf(O.bf16_rn(I), O.bf16_rn(W), pad=(1, 1, 1, 1)), bias=bias, relu=True)
    R32 = O.epilogue(O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)), bias=bias, relu=True)
    assert O.rel_frobenius(got, R16) <= 1e-5
    assert O.rel_frobenius(got, R32) <= 8e-3


CASES = [
    # N, H, W, C, F, KH, KW, stride, dilation, pad
    (1, 8, 8, 64, 64, 3, 3, (1, 1), (1, 1), (1, 1, 1, 1)),
    (2, 13, 11, 16, 24, 3, 3, (2, 1), (1, 2), (1, 0, 2, 1)),
    (1, 12, 12, 5, 7, 3, 3, (1, 1), (1, 1), (0, 0, 0, 0)),      # C not a multiple of 8
    (2, 9, 9, 200, 72, 3, 3, (2, 2), (1, 1), (1, 1, 1, 1)),     # partial channel block
    (3, 7, 7, 128, 96, 1, 1, (1, 1), (1, 1), (0, 0, 0, 0)),     # several images per tile
    (1, 20, 18, 32, 300, 5, 3, (1, 2), (2, 1), (2, 2, 1, 1)),
    (4, 14, 14, 64, 128, 3, 3, (2, 2), (1, 1), (1, 1, 1, 1)),
]


@pytest.mark.parametrize("case", CASES)
def test_bf16_conv_small_ints_bitwise(nk, case):
    N, H, Wd, C, F, KH, KW, st, dl, pad = case
    I = synth.small_ints(81, H * 100 + C, (N, H, Wd, C))
    W = synth.small_ints(81, F * 100 + KH, (KH, KW, C, F))
    np.testing.assert_array_equal(_conv(nk, I, W, st, dl, pad), O.conv2d_nhwc_hwcf(I, W, st, dl, pad))


@pytest.mark.parametrize("sched", [(128, 64, 64, 1, 4, 1), (128, 128, 64, 1, 3, 1), (128, 64, 64, 1, 5, 3),
                                   (128, 256, 64, 1, 4, 2), (256, 128, 64, 2, 4, 1), (256, 64, 64, 2, 6, 3),
                                   (256, 128, 64, 1, 4, 1), (512, 64, 64, 1, 3, 1), (512, 64, 64, 1, 2, 3),
                                   (256, 128, 64, 1, 2, 3), (256, 128, 64, 1, 3, 2)])
def test_bf16_conv_schedules_bitwise(nk, sched):
    N, H, Wd, C, F, KH, KW = 2, 15, 17, 96, 160, 3, 3
    I = synth.small_ints(82, 1, (N, H, Wd, C))
    W = synth.small_ints(82, 2, (KH, KW, C, F))
    got = _conv(nk, I, W, (1, 1), (1, 1), (1, 1, 1, 1), schedule=sched)
    np.testing.assert_array_equal(got, O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)))


def test_bf16_conv_bf16_input_and_accumulate(nk):
    N, H, Wd, C, F = 2, 10, 10, 64, 64
    I = synth.normal(83, 0, (N, H, Wd, C))
    W = synth.normal(83, 1, (3, 3, C, F), sigma=0.06)
    C0 = synth.uniform(83, 2, (N, H, Wd, F))
    out = dev(C0)
    nk.nk_conv2d_nhwc_hwcf(dev(I).to(torch.bfloat16), dev(W), out, pad=(1, 1, 1, 1), precision="bf16",
                           accumulate=True)
    nk.nk_sync_status()
    R = O.epilogue(O.conv2d_nhwc_hwcf(O.bf16_rn(I), O.bf16_rn(W), pad=(1, 1, 1, 1)), c_in=C0, beta=1.0)
    assert O.rel_frobenius(host(out), R) <= 1e-5


@pytest.mark.parametrize("batch", [1, 8])
def test_bf16_resnet_stack_layers(nk, batch):
    for li, L in enumerate(synth.resnet_stack(batch)):
        if li % 3:      # a third of the layers keeps the oracle quick
            continue
        I = synth.half_normal(84, li, (L["N"], L["H"], L["W"], L["C"]))
        W = synth.normal(84, 100 + li, (L["KH"], L["KW"], L["C"], L["F"]),
                         sigma=float(np.sqrt(2.0 / (L["KH"] * L["KW"] * L["C"]))))
        st, pad = (L["stride"],) * 2, (L["pad"],) * 4
        got = _conv(nk, I, W, st, (1, 1), pad)
        R = O.conv2d_nhwc_hwcf(O.bf16_rn(I), O.bf16_rn(W), st, (1, 1), pad)
        assert O.rel_frobenius(got, R) <= 1e-5, (li, L)


WINDOW_CASES = [
    # N, H, W, C, F, KH, KW, dilation, pad  (stride 1)
    (1, 8, 8, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),
    (2, 13, 11, 16, 24, 3, 3, (1, 2), (1, 0, 2, 1)),
    (1, 12, 12, 5, 7, 3, 3, (1, 1), (0, 0, 0, 0)),       # C not a multiple of 8
    (2, 9, 9, 200, 72, 3, 3, (1, 1), (1, 1, 1, 1)),      # partial channel block, weights streamed
    (1, 20, 18, 32, 300, 5, 3, (2, 1), (2, 2, 1, 1)),    # several N tiles, dilation
    (5, 7, 7, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),       # several images per window
    (1, 6, 140, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),     # rows wider than one window
    (2, 15, 17, 96, 160, 3, 3, (1, 1), (1, 1, 1, 1)),
]
WINDOW_SCHEDULES = [  # tile_m, tile_n, stages
    (128, 64, 2), (128, 128, 1), (128, 256, 3), (256, 64, 2), (256, 128, 2), (512, 64, 2), (512, 64, 1),
    (128, 64, 4), (128, 64, 1), (256, 64, 1)]


@pytest.mark.parametrize("case", WINDOW_CASES)
@pytest.mark.parametrize("ws", WINDOW_SCHEDULES)
def test_bf16_conv_window_bitwise(nk, case, ws):
    """Stride-1 conv from one shared input window per tile: every tap reads
    the window from a row offset (tile_k = 64 * taps selects this path)."""
    N, H, Wd, C, F, KH, KW, dl, pad = case
    tm, tn, stages = ws
    I = synth.small_ints(86, H * 100 + C, (N, H, Wd, C))
    W = synth.small_ints(86, F * 100 + KH, (KH, KW, C, F))
    sched = (tm, tn, 64 * KH * KW, 1, stages, 1)
    got = _conv(nk, I, W, (1, 1), dl, pad, schedule=sched)
    np.testing.assert_array_equal(got, O.conv2d_nhwc_hwcf(I, W, (1, 1), dl, pad))


def test_bf16_conv_window_epilogue(nk):
    """Bias, ReLU and accumulate through the window kernel, BF16 input."""
    N, H, Wd, C, F = 3, 19, 23, 64, 96
    I = synth.normal(87, 0, (N, H, Wd, C))
    W = synth.normal(87, 1, (3, 3, C, F), sigma=0.06)
    bias = synth.uniform(87, 2, (F,), lo=-0.1, hi=0.1)
    C0 = synth.uniform(87, 3, (N, H, Wd, F))
    out = dev(C0)
    nk.nk_conv2d_nhwc_hwcf(dev(I).to(torch.bfloat16), dev(W), out, pad=(1, 1, 1, 1), precision="bf16",
                           bias=dev(bias), relu=True, accumulate=True, schedule=(256, 128, 576, 1, 2, 1))
    nk.nk_sync_status()
    R = O.epilogue(O.conv2d_nhwc_hwcf(O.bf16_rn(I), O.bf16_rn(W), pad=(1, 1, 1, 1)), c_in=C0, beta=1.0,
                   bias=bias, relu=True)
    assert O.rel_frobenius(host(out), R) <= 1e-5


def test_bf16_conv_window_rejects_strided(nk):
    """The window path is stride 1 only; a strided problem with its tile_k is
    refused before launch."""
    I = synth.small_ints(88, 0, (1, 9, 9, 64))
    W = synth.small_ints(88, 1, (3, 3, 64, 64))
    with pytest.raises(nk.NkError):
        _conv(nk, I, W, (2, 2), (1, 1), (1, 1, 1, 1), schedule=(128, 64, 576, 1, 2, 1))


@pytest.mark.parametrize("case", [(2, 11, 13, 64, 96, 3, 3, 1), (1, 9, 9, 20, 40, 3, 3, 1), (2, 10, 10, 72, 64, 3, 3, 2),
                                  (1, 7, 7, 128, 80, 1, 1, 1)])
@pytest.mark.parametrize("path", ["window", "tap"])
def test_bf16_conv_packed_weights_bitwise(nk, case, path):
    """Weights packed once by nk_conv2d_pack_weights (BF16, channels
    contiguous per filter tap) give the same bits as FP32 weights converted
    per call, on both kernels."""
    N, H, Wd, C, F, KH, KW, s = case
    if path == "window" and (s != 1 or KH * KW == 1):
        pytest.skip("the window kernel is for stride-1 multi-tap convolutions")
    I = synth.small_ints(89, H * 100 + C, (N, H, Wd, C))
    W = synth.small_ints(89, F * 100 + KH, (KH, KW, C, F))
    sched = (128, 64, 64 * KH * KW if path == "window" else 64, 1, 2, 1)
    pad = (KH // 2,) * 4
    ref = _conv(nk, I, W, (s, s), (1, 1), pad, schedule=sched)
    Wp = nk.nk_conv2d_pack_weights(dev(W))
    assert Wp.dtype == torch.bfloat16 and Wp.stride(2) == 1 and Wp.stride(1) % 8 == 0
    N_, OH, OW = N, ref.shape[1], ref.shape[2]
    out = torch.empty(N_, OH, OW, F, device=DEV)
    # FP32 I: converted (channels padded to 8) in the workspace, beside the packed BF16 W
    nk.nk_conv2d_nhwc_hwcf(dev(I), Wp, out, stride=(s, s), pad=pad, precision="bf16", schedule=sched)
    nk.nk_sync_status()
    np.testing.assert_array_equal(host(out), ref)
    np.testing.assert_array_equal(ref, O.conv2d_nhwc_hwcf(I, W, (s, s), (1, 1), pad))


def test_bf16_conv_rejects_unpacked_bf16_weights(nk):
    """A BF16 W in plain HWCF order (F innermost) is not the packed layout."""
    I = synth.small_ints(90, 0, (1, 8, 8, 64))
    W = synth.small_ints(90, 1, (3, 3, 64, 64))
    out = torch.empty(1, 8, 8, 64, device=DEV)
    with pytest.raises(nk.NkError):
        nk.nk_conv2d_nhwc_hwcf(dev(I).to(torch.bfloat16), dev(W).to(torch.bfloat16), out, pad=(1, 1, 1, 1),
                               precision="bf16")


def _half_ints(seed, stream, shape, edge):
    """Half-integers in [-2, 2] with one entry = edge (|edge| = 3.5 = amax):
    the E4M3 scale 448 / 3.5 = 128 is exact and every value x*128 is an
    E4M3 code, so the quantised convolution is exact."""
    x = synth.small_ints(seed, stream, shape) / 2
    x.flat[0] = edge
    return x


FP8_CASES = [
    # N, H, W, C, F, KH, KW, stride, dilation, pad
    (1, 8, 8, 64, 64, 3, 3, (1, 1), (1, 1), (1, 1, 1, 1)),
    (2, 13, 11, 20, 24, 3, 3, (2, 1), (1, 2), (1, 0, 2, 1)),     # C = 20: rows padded to 32 bytes
    (2, 9, 9, 200, 72, 3, 3, (2, 2), (1, 1), (1, 1, 1, 1)),     # two 128-channel K blocks per tap
    (3, 7, 7, 128, 96, 1, 1, (1, 1), (1, 1), (0, 0, 0, 0)),
]


@pytest.mark.parametrize("case", FP8_CASES)
@pytest.mark.parametrize("sched", [None, (128, 64, 128, 1, 3, 1), (128, 128, 128, 1, 4, 1), (256, 64, 128, 1, 3, 1),
                                   (512, 64, 128, 1, 2, 1), (128, 128, 128, 1, 3, 3)])
def test_fp8_conv_exact_codes_bitwise(nk, case, sched):
    """E4M3 convolution with per-tensor amax scales (s_i, s_w), dequantised by
    1/(s_i*s_w) in the epilogue; on exactly representable inputs it equals
    the FP64 oracle bit for bit."""
    N, H, Wd, C, F, KH, KW, st, dl, pad = case
    I = _half_ints(97, H * 100 + C, (N, H, Wd, C), 3.5)
    W = _half_ints(97, F * 100 + KH, (KH, KW, C, F), -3.5)
    OH = O.conv_out_size(H, KH, st[0], dl[0], pad[0], pad[1])
    OW = O.conv_out_size(Wd, KW, st[1], dl[1], pad[2], pad[3])
    out = torch.empty(N, OH, OW, F, device=DEV)
    nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), out, stride=st, dilation=dl, pad=pad, precision="fp8", schedule=sched)
    nk.nk_sync_status()
    np.testing.assert_array_equal(host(out), O.conv2d_nhwc_hwcf(I, W, st, dl, pad))


def test_fp8_conv_resnet_block_tolerance(nk):
    """The FP32 conv config in E4M3: within 6e-2 of the FP32 result, and
    within 1e-5 of the exact convolution of the dequantised E4M3 operands."""
    I, W, bias = synth.conv_resnet_block()
    out = torch.empty(8, 56, 56, 64, device=DEV)
    nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), out, pad=(1, 1, 1, 1), precision="fp8", bias=dev(bias), relu=True)
    nk.nk_sync_status()
    got = host(out)
    R32 = O.epilogue(O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)), bias=bias, relu=True)
    assert O.rel_frobenius(got, R32) <= 6e-2
    si, sw = O.fp8_scale(I), O.fp8_scale(W)
    Rq = O.conv2d_nhwc_hwcf(O.fp8_quantize(I, si), O.fp8_quantize(W, sw), pad=(1, 1, 1, 1))
    Rq = O.epilogue(Rq / (np.float64(si) * np.float64(sw)), bias=bias, relu=True)
    assert O.rel_frobenius(got, Rq) <= 1e-5


def test_fp8_conv_rejects_pairs_and_bf16_input(nk):
    I = synth.small_ints(98, 0, (1, 8, 8, 64))
    W = synth.small_ints(98, 1, (3, 3, 64, 64))
    out = torch.empty(1, 8, 8, 64, device=DEV)
    for sched in [(256, 64, 128, 2, 3, 1), (128, 64, 128, 2, 3, 1)]:
        with pytest.raises(nk.NkError):
            nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), out, pad=(1, 1, 1, 1), precision="fp8", schedule=sched)
    with pytest.raises(nk.NkError):
        nk.nk_conv2d_nhwc_hwcf(dev(I).to(torch.bfloat16), dev(W), out, pad=(1, 1, 1, 1), precision="fp8")


@pytest.mark.parametrize("case", [(2, 9, 11, 64, 40, 3, 3, (1, 1), (1, 1), (1, 1, 1, 1)),
                                  (1, 12, 10, 24, 72, 3, 3, (2, 1), (1, 2), (0, 1, 2, 0))])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_gpu_conv_equals_gpu_gemm_on_explicit_im2col(nk, case, prec):
    """The GPU convolution equals the GPU GEMM on an explicit im2col matrix
    (built by the oracle's separate patch code) and the FP64 definition."""
    N, H, Wd, C, F, KH, KW, st, dl, pad = case
    if prec == "fp8":
        I = _half_ints(99, H + C, (N, H, Wd, C), 3.5)
        W = _half_ints(99, F + KH, (KH, KW, C, F), 3.5)
    else:
        I = synth.small_ints(99, H + C, (N, H, Wd, C))
        W = synth.small_ints(99, F + KH, (KH, KW, C, F))
    conv = _conv(nk, I, W, st, dl, pad) if prec == "bf16" else None
    if conv is None:
        OH = O.conv_out_size(H, KH, st[0], dl[0], pad[0], pad[1])
        OW = O.conv_out_size(Wd, KW, st[1], dl[1], pad[2], pad[3])
        out = torch.empty(N, OH, OW, F, device=DEV)
        nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), out, stride=st, dilation=dl, pad=pad, precision="fp8")
        nk.nk_sync_status()
        conv = host(out)
    P = O.im2col(I, KH, KW, st, dl, pad).astype(np.float32)
    Wm = W.reshape(KH * KW * C, F)
    c = torch.empty(P.shape[0], F, device=DEV)
    nk.nk_matmul(dev(P), dev(Wm), c, precision=prec)
    nk.nk_sync_status()
    gemm = host(c).reshape(conv.shape)
    np.testing.assert_array_equal(conv, gemm)
    np.testing.assert_array_equal(conv, O.conv2d_nhwc_hwcf(I, W, st, dl, pad))


CONV_GROUPS = [
    # N, H, W, C, F, KH, KW, stride, dilation, pad, relu, accumulate
    (2, 14, 14, 64, 64, 3, 3, (1, 1), (1, 1), (1, 1, 1, 1), True, False),
    (1, 9, 13, 128, 96, 3, 3, (2, 2), (1, 1), (1, 1, 1, 1), False, False),
    (3, 7, 7, 64, 200, 1, 1, (1, 1), (1, 1), (0, 0, 0, 0), True, True),
    (1, 20, 18, 32, 40, 5, 3, (1, 2), (2, 1), (2, 2, 1, 1), False, True),
    (2, 5, 6, 16, 24, 3, 3, (1, 1), (1, 1), (0, 1, 2, 0), True, False),
    (1, 30, 30, 8, 8, 3, 3, (1, 1), (1, 1), (1, 1, 1, 1), False, False),
]


def _conv_group_operands(nk, seed):
    convs, refs = [], []
    for i, (N, H, Wd, C, F, KH, KW, st, dl, pad, relu, acc) in enumerate(CONV_GROUPS):
        I = synth.small_ints(seed, 10 * i, (N, H, Wd, C))
        W = synth.small_ints(seed, 10 * i + 1, (KH, KW, C, F))
        b = synth.small_ints(seed, 10 * i + 2, (F,))
        OH = O.conv_out_size(H, KH, st[0], dl[0], pad[0], pad[1])
        OW = O.conv_out_size(Wd, KW, st[1], dl[1], pad[2], pad[3])
        C0 = synth.small_ints(seed, 10 * i + 3, (N, OH, OW, F)) if acc else np.zeros((N, OH, OW, F), np.float32)
        convs.append(dict(I=dev(I).to(torch.bfloat16), W=nk.nk_conv2d_pack_weights(dev(W)), O=dev(C0), stride=st,
                          dilation=dl, pad=pad, bias=dev(b), relu=relu, accumulate=acc))
        refs.append(O.epilogue(O.conv2d_nhwc_hwcf(I, W, st, dl, pad), c_in=C0, beta=1.0 if acc else 0.0, bias=b,
                               relu=relu))
    return convs, refs


@pytest.mark.parametrize("sched", [None, (128, 64, 64, 1, 4, 1), (128, 256, 64, 1, 3, 1)])
def test_grouped_convs_one_launch_bitwise(nk, sched):
    """Six uneven convolutions (strides, dilations, 1x1 / 3x3 / 5x3 filters,
    bias, ReLU, accumulate) computed by one persistent launch."""
    convs, refs = _conv_group_operands(nk, 100)
    groups, G = nk.make_conv_groups(convs)
    plan = nk.nk_conv2d_grouped_plan_create(groups, G, schedule=sched)
    nk.nk_grouped_plan_run(plan)
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)
    for g in range(G):
        np.testing.assert_array_equal(host(convs[g]["O"]), refs[g], err_msg=f"group {g}")


def test_grouped_convs_graph_replay(nk):
    """The grouped conv launch captured in a CUDA graph and replayed gives
    the eager result (accumulate groups excluded: they add on every run)."""
    convs, refs = _conv_group_operands(nk, 101)
    for d in convs:
        d["accumulate"] = False
    groups, G = nk.make_conv_groups(convs)
    plan = nk.nk_conv2d_grouped_plan_create(groups, G)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        nk.nk_grouped_plan_run(plan, s.cuda_stream)
        torch.cuda.synchronize()
        eager = [host(d["O"]).copy() for d in convs]
        for d in convs:
            d["O"].zero_()
        with torch.cuda.graph(g, stream=s):
            nk.nk_grouped_plan_run(plan, s.cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)
    for i in range(G):
        np.testing.assert_array_equal(host(convs[i]["O"]), eager[i])


def test_grouped_convs_reject_bad_groups(nk):
    convs, _ = _conv_group_operands(nk, 102)
    bad = dict(convs[0])
    bad["I"] = bad["I"].float()       # FP32 input: the grouped launch takes BF16
    groups, G = nk.make_conv_groups([convs[1], bad])
    with pytest.raises(nk.NkError):
        nk.nk_conv2d_grouped_plan_create(groups, G)


def test_grouped_convs_tune_and_exact(nk):
    """nk_conv2d_grouped_tune returns the fastest legal grouped-conv tile (no
    slower than the built-in one) and a plan built with it stays exact."""
    from paper_2307_16080_gb300 import nk_tune as nt
    convs, refs = _conv_group_operands(nk, 103)
    groups, G = nk.make_conv_groups(convs)
    best, rep = nt.nk_conv2d_grouped_tune(groups, G, reps=3)
    assert rep.timed == rep.candidates >= 10 and best[0] == 128 and best[3] == 1 and best[5] == 1
    assert 0 < rep.best_ms <= rep.default_ms * 1.05
    convs, refs = _conv_group_operands(nk, 103)     # fresh O (tuning overwrote them)
    groups, G = nk.make_conv_groups(convs)
    plan = nk.nk_conv2d_grouped_plan_create(groups, G, schedule=best)
    nk.nk_grouped_plan_run(plan)
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)
    for g in range(G):
        np.testing.assert_array_equal(host(convs[g]["O"]), refs[g], err_msg=f"group {g}")
