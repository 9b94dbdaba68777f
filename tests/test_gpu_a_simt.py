"""GPU parity of the FP32 CUDA-core path, the operand prep casts and the
validation norm against the FP64 oracle (called through the C ABI)."""
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


def _mm(nk, a, b, M, N, prec="f32", c=None, **kw):
    c = torch.empty(M, N, device=DEV) if c is None else c
    nk.nk_matmul(a, b, c, precision=prec, **kw)
    nk.nk_sync_status()
    return c


def test_f32_matmul_256_config(nk):
    A, B = synth.matmul_uniform(256, 256, 256)
    C = host(_mm(nk, dev(A), dev(B), 256, 256))
    assert O.rel_frobenius(C, O.matmul(A, B)) <= 1e-5


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 7), (17, 31, 33), (64, 64, 16), (127, 129, 65),
                                   (130, 260, 100), (300, 200, 513)])
def test_f32_small_ints_exact(nk, M, N, K):
    A = synth.small_ints(40, M * 7 + K, (M, K))
    B = synth.small_ints(40, N * 11 + K, (K, N))
    C = host(_mm(nk, dev(A), dev(B), M, N))
    np.testing.assert_array_equal(C, O.matmul(A, B))


def test_f32_layouts_and_transpose_identity(nk):
    M, N, K = 96, 80, 72
    A, B = synth.matmul_uniform(M, N, K, seed=41)
    ref = host(_mm(nk, dev(A), dev(B), M, N))
    assert O.rel_frobenius(ref, O.matmul(A, B)) <= 1e-5
    for a in (dev(A), colmajor(A)):
        for b in (dev(B), colmajor(B)):
            c = _mm(nk, a, b, M, N)
            np.testing.assert_array_equal(host(c), ref)
            ct = torch.empty(N, M, device=DEV).t()      # column-major C: C^T = B^T A^T
            _mm(nk, a, b, M, N, c=ct)
            np.testing.assert_array_equal(host(ct), ref)


@pytest.mark.parametrize("split", [1, 2, 4, 7])
def test_f32_epilogue_and_split_k(nk, split):
    M, N, K = 150, 270, 1000
    A, B = synth.matmul_uniform(M, N, K, seed=42)
    C0 = synth.uniform(42, 7, (M, N))
    bias = synth.uniform(42, 8, (N,), -0.5, 0.5)
    R = O.epilogue(O.matmul(A, B), c_in=C0, bias=bias, relu=True, beta=1.0)
    outs = []
    for _ in range(2):
        c = dev(C0)
        _mm(nk, dev(A), dev(B), M, N, c=c, bias=dev(bias), relu=True, accumulate=True,
            schedule=(64, 64, 16, 1, 2, split))
        outs.append(host(c))
    assert O.rel_frobenius(outs[0], R) <= 1e-5
    np.testing.assert_array_equal(outs[0], outs[1])   # fixed-order reduction


def test_f32_conv_resnet_block_config(nk):
    I, W, bias = synth.conv_resnet_block()
    O_ = torch.empty(8, 56, 56, 64, device=DEV)
    nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), O_, stride=(1, 1), pad=(1, 1, 1, 1), bias=dev(bias), relu=True)
    nk.nk_sync_status()
    R = O.epilogue(O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)), bias=bias, relu=True)
    assert O.rel_frobenius(host(O_), R) <= 1e-5


@pytest.mark.parametrize("case", [
    (1, 5, 6, 3, 2, 3, 3, (1, 1), (1, 1), (0, 0, 0, 0)),
    (2, 9, 7, 8, 5, 3, 3, (2, 1), (1, 2), (1, 0, 2, 1)),
    (1, 12, 12, 16, 24, 3, 3, (2, 2), (1, 1), (1, 1, 1, 1)),
    (2, 7, 7, 32, 40, 1, 1, (1, 1), (1, 1), (0, 0, 0, 0)),
    (1, 11, 13, 5, 7, 5, 3, (1, 2), (2, 1), (2, 2, 1, 1)),
])
def test_f32_conv_variants(nk, case):
    N, H, Wd, C, F, KH, KW, st, dl, pad = case
    I = synth.small_ints(43, H * 31 + C, (N, H, Wd, C))
    W = synth.small_ints(43, F * 17 + KH, (KH, KW, C, F))
    R = O.conv2d_nhwc_hwcf(I, W, st, dl, pad)
    O_ = torch.empty(*R.shape, device=DEV)
    nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), O_, stride=st, dilation=dl, pad=pad)
    nk.nk_sync_status()
    np.testing.assert_array_equal(host(O_), R)


def _bit_patterns(n, seed):
    x = synth.raw_u64(seed, 0, n).astype(np.uint32).view(np.float32)
    x = x[np.isfinite(x)]
    return x


def test_prep_bf16_cast_bitwise(nk):
    x = _bit_patterns(1 << 22, 44).reshape(-1)[: (1 << 21)].reshape(1024, -1)
    out = torch.empty(x.shape, dtype=torch.bfloat16, device=DEV)
    nk.nk_cast_bf16(dev(x), out)
    torch.cuda.synchronize()
    got = out.float().cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got, O.bf16_rn(x))
    outT = torch.empty(x.shape[::-1], dtype=torch.bfloat16, device=DEV)
    nk.nk_cast_bf16(dev(x), outT, transpose=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(outT.float().cpu().numpy().T.astype(np.float64), O.bf16_rn(x))


@pytest.mark.parametrize("shape", [(1000, 1536), (333, 77)])
def test_prep_fp8_amax_and_cast_bitwise(nk, shape):
    x = synth.outlier_normal(45, shape[0], shape)
    amax = torch.empty(1, device=DEV)
    nk.nk_amax(dev(x), amax)
    torch.cuda.synchronize()
    assert amax.item() == np.max(np.abs(x))
    s_ref = O.fp8_scale(x)
    q = torch.empty(shape, dtype=torch.uint8, device=DEV)
    s_out = torch.empty(1, device=DEV)
    nk.nk_cast_fp8(dev(x), amax, q, scale_out=s_out)
    torch.cuda.synchronize()
    assert s_out.item() == float(s_ref)
    got = q.view(torch.float8_e4m3fn).float().cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got, O.fp8_quantize(x, s_ref))
    qT = torch.empty(shape[::-1], dtype=torch.uint8, device=DEV)
    nk.nk_cast_fp8(dev(x), amax, qT, transpose=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(qT.view(torch.float8_e4m3fn).float().cpu().numpy().T.astype(np.float64),
                                  O.fp8_quantize(x, s_ref))


def test_prep_fp8_zero_amax_gives_unit_scale(nk):
    x = np.zeros((8, 32), np.float32)
    amax = torch.empty(1, device=DEV)
    nk.nk_amax(dev(x), amax)
    q = torch.empty(x.shape, dtype=torch.uint8, device=DEV)
    s_out = torch.empty(1, device=DEV)
    nk.nk_cast_fp8(dev(x), amax, q, scale_out=s_out)
    torch.cuda.synchronize()
    assert amax.item() == 0.0 and s_out.item() == 1.0 and int(q.sum()) == 0


def test_prep_bf16x3_split_bitwise(nk):
    x = synth.outlier_normal(46, 0, (512, 640))
    hi = torch.empty(x.shape, dtype=torch.bfloat16, device=DEV)
    lo = torch.empty_like(hi)
    nk.nk_split_bf16x3(dev(x), hi, lo)
    torch.cuda.synchronize()
    rh, rl = O.bf16x3_split(x)
    np.testing.assert_array_equal(hi.float().cpu().numpy().astype(np.float64), rh)
    np.testing.assert_array_equal(lo.float().cpu().numpy().astype(np.float64), rl)


def test_validation_norm_fp64(nk):
    C = synth.normal(47, 0, (777, 513))
    R = C.astype(np.float64) + synth.normal(47, 1, (777, 513)).astype(np.float64) * 1e-3
    out = nk.nk_rel_frobenius(dev(C), dev(R, torch.float64))
    torch.cuda.synchronize()
    e, r2 = out.cpu().numpy()
    assert abs(e - np.sum((C - R) ** 2)) <= 1e-10 * e
    assert abs(r2 - np.sum(R ** 2)) <= 1e-12 * r2
    out2 = nk.nk_rel_frobenius(dev(C), dev(R, torch.float64))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), out2.cpu().numpy())


def test_bad_arguments_return_status(nk):
    a = torch.empty(4, 5, device=DEV)
    b = torch.empty(6, 7, device=DEV)
    c = torch.empty(4, 7, device=DEV)
    with pytest.raises(nk.NkError) as e:
        nk.nk_matmul(a, b, c)
    assert e.value.status == -1
    with pytest.raises(nk.NkError) as e:   # split-K without workspace
        ta, tb, tc = nk.as_nk_tensor(a), nk.as_nk_tensor(torch.empty(5, 7, device=DEV)), nk.as_nk_tensor(c)
        s = nk.nk_schedule(64, 64, 16, 1, 2, 4)
        st = nk.lib().nk_matmul(nk.ctypes.byref(ta), nk.ctypes.byref(tb), nk.ctypes.byref(tc), 0, None,
                                nk.ctypes.byref(s), None, 0, 0)
        nk._check(st)
    assert e.value.status == -4
