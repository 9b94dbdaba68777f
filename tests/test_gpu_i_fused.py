"""GPU parity of the fused elementwise programs (epilogues on C / O, prologues
on the FP32 operands, and the standalone elementwise pass) against the FP64
oracle, through the C ABI.

Tolerances (relative Frobenius unless stated):
* FP32, BF16x3 and BF16-vs-rounded-inputs keep their contract bounds (1e-5,
  2e-5, 1e-5) whenever the prologue is exact in FP32 (mul, add, affine, relu,
  clamp): device and oracle then round the same FP32 value.
* A transcendental prologue (gelu, tanh, ...) is evaluated by CUDA's FP32
  functions on the device and in FP64 then rounded to FP32 by the oracle; the
  two FP32 values can differ by a few ulps, which flips the BF16 rounding of a
  fraction p ~ 4 * 2^-16 of the operand elements, each by one BF16 ulp
  (2^-8 relative).  The contraction then differs by ~ sqrt(p) * 2^-8 ~ 3e-5
  relative; the bound used is 1e-4 (and 8e-3 against the FP32 inputs).
* The standalone pass is checked per element: 3e-5 relative (the argument
  rounding of erfc / exp at |x| <= 8 amplifies to a few 1e-6).
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import DEV, colmajor, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


def _programs(shape, seed):
    T1 = synth.normal(seed, 10, shape).astype(np.float32)
    T2 = synth.uniform(seed, 11, shape).astype(np.float32)
    return {
        "mul": [("mul", T1)],
        "add_relu": [("add", T1), ("relu",)],
        "affine_clamp": [("affine", 0.75, -0.25), ("clamp", -0.5, 0.5)],
        "gelu": [("gelu",)],
        "gelu_tanh_mul": [("gelu_tanh",), ("mul", T2)],
        "silu_add": [("silu",), ("add", T1)],
        "sigmoid": [("sigmoid",)],
        "tanh_affine": [("tanh",), ("affine", 2.0, 1.0)],
        "four_steps": [("affine", 0.5, 0.1), ("gelu",), ("mul", T1), ("add", T2)],
    }


PROGRAM_NAMES = list(_programs((1, 1), 0))


def _dev_prog(prog, layout=dev):
    """The same program with its tensor operands on the device, laid out by
    `layout` (dev: row-major, colmajor: column-major)."""
    if prog is None:
        return None
    return [(s[0], layout(s[1])) if s[0] in ("mul", "add") else s for s in prog]


def _mm(nk, A, B, prec, C=None, **kw):
    M, N = A.shape[0], B.shape[1]
    C = torch.empty(M, N, device=DEV) if C is None else C
    nk.nk_matmul(dev(A), dev(B), C, prec, **kw)
    nk.nk_sync_status()
    return host(C)


# ---------------------------------------------------------------- matmul epilogues
@pytest.mark.parametrize("name", PROGRAM_NAMES)
def test_f32_epilogue_program(nk, name):
    M, N, K = 200, 136, 72
    A, B = synth.matmul_uniform(M, N, K, seed=70)
    bias = synth.uniform(70, 3, (N,)).astype(np.float32)
    prog = _programs((M, N), 71)[name]
    got = _mm(nk, A, B, "f32", bias=dev(bias), ew=_dev_prog(prog))
    want = O.matmul_fused(A, B, "f32", bias=bias, ew=prog)
    assert O.rel_frobenius(got, want) <= 1e-5


@pytest.mark.parametrize("name", PROGRAM_NAMES)
def test_bf16_epilogue_program(nk, name):
    M, N, K = 300, 264, 256
    A, B = synth.matmul_outlier(M, N, K, seed=72)
    prog = _programs((M, N), 73)[name]
    got = _mm(nk, A, B, "bf16", relu=(name == "gelu"), ew=_dev_prog(prog))
    # against the contraction of the bf16-rounded operands; a program that
    # saturates (clamp, sigmoid) changes what "relative to FP32" measures, so
    # the 8e-3 bound of the contraction is not restated after it
    assert O.rel_frobenius(got, O.matmul_fused(A, B, "bf16", relu=(name == "gelu"), ew=prog)) <= 1e-5


def test_fp8_and_bf16x3_epilogue_program(nk):
    M, N, K = 256, 200, 192
    A, B = synth.matmul_outlier(M, N, K, seed=74)
    prog = _programs((M, N), 75)["four_steps"]
    R32 = O.matmul_fused(A, B, "f32", ew=prog)
    got = _mm(nk, A, B, "fp8", ew=_dev_prog(prog))
    assert O.rel_frobenius(got, R32) <= 6e-2
    assert O.rel_frobenius(got, O.matmul_fused(A, B, "fp8", ew=prog)) <= 1e-5
    got = _mm(nk, A, B, "bf16x3", ew=_dev_prog(prog))
    assert O.rel_frobenius(got, R32) <= 2e-5


# ---------------------------------------------------------------- matmul prologues
PROLOGUES = {
    "exact": ([("relu",)], [("affine", 2.0, -0.5)]),
    "tensor": ("mul_a", [("clamp", -1.0, 1.0)]),
    "transcendental": ([("gelu",)], [("tanh",)]),
}


def _prologues(kind, A, B, seed):
    pa, pb = PROLOGUES[kind]
    if pa == "mul_a":
        pa = [("mul", synth.uniform(seed, 20, A.shape).astype(np.float32)), ("add", synth.normal(seed, 21, A.shape).astype(np.float32))]
    return pa, pb


@pytest.mark.parametrize("kind", list(PROLOGUES))
@pytest.mark.parametrize("prec", ["f32", "bf16", "fp8", "bf16x3"])
def test_prologues(nk, prec, kind):
    M, N, K = 264, 136, 200
    A, B = synth.matmul_outlier(M, N, K, seed=76)
    pa, pb = _prologues(kind, A, B, 77)
    got = _mm(nk, A, B, prec, pro_a=_dev_prog(pa), pro_b=_dev_prog(pb))
    R32 = O.matmul_fused(A, B, "f32", pro_a=pa, pro_b=pb)
    exact = kind != "transcendental"
    if prec == "f32":
        assert O.rel_frobenius(got, R32) <= 1e-5
    elif prec == "bf16":
        assert O.rel_frobenius(got, O.matmul_fused(A, B, "bf16", pro_a=pa, pro_b=pb)) <= (1e-5 if exact else 1e-4)
        assert O.rel_frobenius(got, R32) <= 8e-3
    elif prec == "fp8":
        assert O.rel_frobenius(got, R32) <= 6e-2
        if exact:
            assert O.rel_frobenius(got, O.matmul_fused(A, B, "fp8", pro_a=pa, pro_b=pb)) <= 1e-5
    else:
        assert O.rel_frobenius(got, R32) <= 2e-5


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_layouts_column_major_c_and_operands(nk, prec):
    """C column-major swaps the operands (C^T = B^T A^T) and with them the
    prologues; column-major A / B take the transposing cast.  Tensor
    operands follow the layout of the tensor they pair with."""
    M, N, K = 136, 200, 96
    A, B = synth.matmul_outlier(M, N, K, seed=78)
    TA = synth.uniform(78, 5, (M, K)).astype(np.float32)
    TC = synth.normal(78, 6, (M, N)).astype(np.float32)
    pa = [("mul", TA), ("relu",)]
    pb = [("affine", 0.5, 0.0)]
    ew = [("add", TC), ("silu",)]
    want = O.matmul_fused(A, B, prec, pro_a=pa, pro_b=pb, ew=ew)
    for a_l, b_l, c_l in [(dev, dev, colmajor), (colmajor, dev, dev), (dev, colmajor, colmajor),
                          (colmajor, colmajor, dev)]:
        C = c_l(np.zeros((M, N), np.float32))
        nk.nk_matmul(a_l(A), b_l(B), C, prec, pro_a=_dev_prog(pa, a_l), pro_b=_dev_prog(pb, b_l),
                     ew=_dev_prog(ew, c_l))
        nk.nk_sync_status()
        assert O.rel_frobenius(host(C), want) <= 1e-5, (a_l.__name__, b_l.__name__, c_l.__name__)


def test_f32_scalar_load_modes_with_prologue(nk):
    # K and strides not multiples of 4: the scalar A / B load paths
    M, N, K = 70, 53, 37
    A, B = synth.matmul_uniform(M, N, K, seed=79)
    Abig = torch.zeros(M, K + 3, device=DEV)
    Abig[:, :K] = dev(A)
    a = Abig[:, :K]
    TA = synth.normal(79, 7, (M, K)).astype(np.float32)
    TAbig = torch.zeros(M, K + 3, device=DEV)
    TAbig[:, :K] = dev(TA)
    C = torch.empty(M, N, device=DEV)
    nk.nk_matmul(a, dev(B), C, "f32", pro_a=[("add", TAbig[:, :K])], pro_b=[("sigmoid",)])
    nk.nk_sync_status()
    want = O.matmul_fused(A, B, "f32", pro_a=[("add", TA)], pro_b=[("sigmoid",)])
    assert O.rel_frobenius(host(C), want) <= 1e-5


# ---------------------------------------------------------------- special paths
@pytest.mark.parametrize("prec,sched", [("bf16", (128, 128, 64, 1, 4, 4)), ("f32", (64, 64, 16, 1, 2, 3)),
                                        ("fp8", (128, 128, 128, 1, 4, 2))])
def test_split_k_applies_program_in_the_reduce(nk, prec, sched):
    M, N, K = 200, 264, 1024
    A, B = synth.matmul_outlier(M, N, K, seed=80)
    prog = _programs((M, N), 81)["four_steps"]
    got = _mm(nk, A, B, prec, ew=_dev_prog(prog), schedule=sched)
    tol = {"bf16": 1e-5, "f32": 1e-5, "fp8": 1e-5}[prec]
    assert O.rel_frobenius(got, O.matmul_fused(A, B, prec, ew=prog)) <= tol


def test_empty_reduction_runs_the_program(nk):
    M, N = 40, 72
    C0 = synth.normal(82, 0, (M, N)).astype(np.float32)
    bias = synth.uniform(82, 1, (N,)).astype(np.float32)
    prog = [("gelu",), ("affine", -1.0, 0.5)]
    for prec in ("f32", "bf16"):
        C = dev(C0)
        nk.nk_matmul(torch.empty(M, 0, device=DEV), torch.empty(0, N, device=DEV), C, prec, bias=dev(bias),
                     accumulate=True, ew=prog)
        nk.nk_sync_status()
        want = O.ew_program(O.epilogue(np.zeros((M, N)), C0, bias, beta=1.0), prog)
        assert O.rel_frobenius(host(C), want) <= 1e-6


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_epilogue_operand_may_alias_the_output(nk, prec):
    M, N, K = 136, 128, 64
    A, B = synth.matmul_uniform(M, N, K, seed=83)
    C0 = synth.normal(83, 2, (M, N)).astype(np.float32)
    C = dev(C0)
    nk.nk_matmul(dev(A), dev(B), C, prec, accumulate=True, ew=[("add", C)])
    nk.nk_sync_status()
    want = O.matmul_fused(A, B, prec, c_in=C0, beta=1.0, ew=[("add", C0)])
    assert O.rel_frobenius(host(C), want) <= 1e-5


def test_large_default_schedule_with_program(nk):
    """A program turns the plain GEMM's TMA-store epilogue into the per-lane
    stores; checked on the built-in schedule of a large problem."""
    M, N, K = 2048, 2048, 512
    A, B = synth.matmul_outlier(M, N, K, seed=84)
    R = synth.normal(84, 9, (M, N)).astype(np.float32)
    prog = [("gelu",), ("add", R)]
    got = _mm(nk, A, B, "bf16", ew=_dev_prog(prog))
    assert O.rel_frobenius(got, O.matmul_fused(A, B, "bf16", ew=prog)) <= 1e-5


# ---------------------------------------------------------------- convolutions
def _conv(nk, I, W, prec, pad, stride=(1, 1), packed=False, **kw):
    N, H, Wd, C = I.shape
    KH, KW, _, F = W.shape
    OH = O.conv_out_size(H, KH, stride[0], 1, pad[0], pad[1])
    OW = O.conv_out_size(Wd, KW, stride[1], 1, pad[2], pad[3])
    out = torch.zeros(N, OH, OW, F, device=DEV)
    w = nk.nk_conv2d_pack_weights(dev(W)) if packed else dev(W)
    i = dev(I).to(torch.bfloat16) if kw.pop("i_bf16", False) else dev(I)
    nk.nk_conv2d_nhwc_hwcf(i, w, out, stride=stride, pad=pad, precision=prec, **kw)
    nk.nk_sync_status()
    return host(out)


def test_conv_f32_prologues_and_epilogue(nk):
    I = synth.normal(85, 0, (4, 12, 13, 16))
    W = synth.normal(85, 1, (3, 3, 16, 24), sigma=0.1)
    R = synth.normal(85, 2, (4, 12, 13, 24)).astype(np.float32)
    pi, pw, ew = [("affine", 0.5, 0.25)], [("tanh",)], [("add", R), ("relu",)]
    got = _conv(nk, I, W, "f32", (1, 1, 1, 1), pro_i=_dev_prog(pi), pro_w=_dev_prog(pw), ew=_dev_prog(ew))
    want = O.conv2d_fused(I, W, "f32", pad=(1, 1, 1, 1), pro_i=pi, pro_w=pw, ew=ew)
    assert O.rel_frobenius(got, want) <= 1e-5


def test_conv_bf16_window_residual_block(nk):
    """The ResNet basic-block tail in one kernel: relu(conv + bias + identity)."""
    I, W, bias = synth.conv_resnet_block(N=2, H=28, W=28)
    Rsd = synth.half_normal(86, 3, I.shape).astype(np.float32)
    ew = [("add", Rsd), ("relu",)]
    got = _conv(nk, I, W, "bf16", (1, 1, 1, 1), packed=True, i_bf16=True, bias=dev(bias), ew=_dev_prog(ew),
                schedule=(128, 64, 576, 1, 1, 1))
    want = O.conv2d_fused(I, W, "bf16", pad=(1, 1, 1, 1), bias=bias, ew=ew)
    assert O.rel_frobenius(got, want) <= 1e-5


def test_conv_bf16_per_tap_prologues(nk):
    # C = 20: the BF16 copies pad channels to 24, so W is packed tap by tap
    I = synth.normal(87, 0, (2, 17, 15, 20))
    W = synth.normal(87, 1, (3, 3, 20, 72), sigma=0.1)
    pi, pw, ew = [("relu",)], [("affine", 2.0, 0.0)], [("gelu",)]
    got = _conv(nk, I, W, "bf16", (1, 1, 1, 1), stride=(2, 2), pro_i=_dev_prog(pi), pro_w=_dev_prog(pw),
                ew=_dev_prog(ew))
    want = O.conv2d_fused(I, W, "bf16", stride=(2, 2), pad=(1, 1, 1, 1), pro_i=pi, pro_w=pw, ew=ew)
    assert O.rel_frobenius(got, want) <= 1e-5


def test_conv_fp8_prologue_sets_the_scale(nk):
    I = synth.half_normal(88, 0, (2, 10, 10, 32))
    W = synth.normal(88, 1, (3, 3, 32, 32), sigma=0.08)
    pi = [("affine", 0.5, 0.0)]
    got = _conv(nk, I, W, "fp8", (1, 1, 1, 1), pro_i=_dev_prog(pi))
    assert O.rel_frobenius(got, O.conv2d_fused(I, W, "fp8", pad=(1, 1, 1, 1), pro_i=pi)) <= 1e-5
    assert O.rel_frobenius(got, O.conv2d_fused(I, W, "f32", pad=(1, 1, 1, 1), pro_i=pi)) <= 6e-2


def test_conv_split_k_program(nk):
    I = synth.normal(89, 0, (1, 7, 7, 256))
    W = synth.normal(89, 1, (3, 3, 256, 128), sigma=0.03)
    ew = [("sigmoid",)]
    got = _conv(nk, I, W, "bf16", (1, 1, 1, 1), ew=ew, schedule=(128, 64, 64, 1, 4, 4))
    assert O.rel_frobenius(got, O.conv2d_fused(I, W, "bf16", pad=(1, 1, 1, 1), ew=ew)) <= 1e-5


@pytest.mark.parametrize("k", [3, 5])
def test_direct_nchw_conv_program(nk, k):
    inp = synth.normal(90, 0, (2, 1, 40, 70))
    ker = synth.normal(90, 1, (3, 1, k, k))
    HO, WO = 40 - k + 1, 70 - k + 1
    T = synth.uniform(90, 2, (2, 3, HO, WO)).astype(np.float32)
    out = torch.empty(2, 3, HO, WO, device=DEV)
    nk.nk_conv2d_nchw_fchw(dev(inp), dev(ker), out, ew=[("sigmoid",), ("mul", dev(T))])
    nk.nk_sync_status()
    ref = O.conv2d_nhwc_hwcf(inp.transpose(0, 2, 3, 1), ker.transpose(2, 3, 1, 0)).transpose(0, 3, 1, 2)
    want = O.ew_program(ref, [("sigmoid",), ("mul", T)])
    assert O.rel_frobenius(host(out), want) <= 1e-5


# ---------------------------------------------------------------- standalone pass
def _close(got, want, rtol=3e-5):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    both_nan = np.isnan(got) & np.isnan(want)
    err = np.abs(got - want)
    ok = both_nan | (err <= rtol * np.abs(want) + 1e-37)
    assert ok.all(), (got[~ok][:5], want[~ok][:5])


def test_elementwise_gpumodule_product_is_exact(nk):
    A = synth.normal(91, 0, (37, 53)).astype(np.float32)
    B = synth.normal(91, 1, (37, 53)).astype(np.float32)
    C = torch.empty(37, 53, device=DEV)
    nk.nk_elementwise(dev(A), C, [("mul", dev(B))])
    nk.nk_sync_status()
    np.testing.assert_array_equal(host(C), A * B)   # one IEEE rounding, as NumPy's FP32 product


@pytest.mark.parametrize("name", PROGRAM_NAMES)
def test_elementwise_programs(nk, name):
    shape = (37, 53)
    X = synth.normal(92, 0, shape, sigma=2.0).astype(np.float32)
    prog = _programs(shape, 93)[name]
    Y = torch.empty(*shape, device=DEV)
    nk.nk_elementwise(dev(X), Y, _dev_prog(prog))
    nk.nk_sync_status()
    want = O.ew_program(X, prog)
    assert O.rel_frobenius(host(Y), want) <= 1e-6
    if name in ("mul", "add_relu", "affine_clamp", "gelu", "sigmoid"):   # no cancellation after the last rounding
        _close(host(Y), want)


def test_elementwise_layouts_in_place_and_ranks(nk):
    X = synth.normal(94, 0, (24, 40), sigma=2.0).astype(np.float32)
    T = synth.uniform(94, 1, (24, 40)).astype(np.float32)
    prog = [("silu",), ("mul", T)]
    want = O.ew_program(X, prog)
    # Y column-major (strided path), T with Y's layout
    Y = colmajor(np.zeros((24, 40), np.float32))
    nk.nk_elementwise(dev(X), Y, _dev_prog(prog, colmajor))
    nk.nk_sync_status()
    assert O.rel_frobenius(host(Y), want) <= 1e-6
    # in place
    Xd = dev(X)
    nk.nk_elementwise(Xd, Xd, _dev_prog(prog))
    nk.nk_sync_status()
    assert O.rel_frobenius(host(Xd), want) <= 1e-6
    # rank 1 (ragged length) and rank 4
    x1 = synth.normal(94, 2, (1001,)).astype(np.float32)
    y1 = torch.empty(1001, device=DEV)
    nk.nk_elementwise(dev(x1), y1, [("gelu",)])
    x4 = synth.normal(94, 3, (2, 3, 5, 7)).astype(np.float32)
    y4 = torch.empty(2, 3, 5, 7, device=DEV)
    nk.nk_elementwise(dev(x4), y4, [("tanh",)])
    nk.nk_sync_status()
    _close(host(y1), O.ew_program(x1, [("gelu",)]))
    _close(host(y4), O.ew_program(x4, [("tanh",)]))
    # empty tensors and an empty program (a copy)
    nk.nk_elementwise(torch.empty(0, 5, device=DEV), torch.empty(0, 5, device=DEV), [("relu",)])
    y = torch.empty(24, 40, device=DEV)
    nk.nk_elementwise(dev(X), y, [])
    nk.nk_sync_status()
    np.testing.assert_array_equal(host(y), X)
