"""GPU parity of the tcgen05 tensor-core matmul (BF16, FP8 E4M3, BF16x3)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import DEV, colmajor, dev, host

pytestmark = pytest.mark.gpu
TOL = {"bf16": 8e-3, "bf16x3": 2e-5, "fp8": 6e-2}   # vs the FP32 inputs


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


def _mm(nk, a, b, M, N, prec, c=None, **kw):
    c = torch.empty(M, N, device=DEV) if c is None else c
    nk.nk_matmul(a, b, c, precision=prec, **kw)
    nk.nk_sync_status()
    return c


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (200, 300, 100), (1, 1, 1), (384, 512, 2048)])
def test_all_ones_closed_form(nk, prec, M, N, K):
    C = host(_mm(nk, dev(np.ones((M, K), np.float32)), dev(np.ones((K, N), np.float32)), M, N, prec))
    if prec == "fp8":   # dequantisation multiplies by the FP32 reciprocal of s_a*s_b
        np.testing.assert_allclose(C, K, rtol=2e-7)
    else:
        np.testing.assert_array_equal(C, K)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "fp8"])
@pytest.mark.parametrize("M,N,K", [(7, 9, 17), (129, 257, 65), (256, 512, 1024), (300, 100, 520)])
def test_small_ints_bitwise(nk, prec, M, N, K):
    A = synth.small_ints(60, M + K, (M, K))
    B = synth.small_ints(60, N + 2 * K, (K, N))
    if prec == "fp8":   # half-integers up to 3.5 with amax 3.5: s = 128, exact codes
        A, B = A / 2, B / 2
        A.flat[0], B.flat[0] = 3.5, -3.5
    C = host(_mm(nk, dev(A), dev(B), M, N, prec))
    np.testing.assert_array_equal(C, O.matmul_precision(A, B, prec))


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
def test_outlier_precision_bounds(nk, prec):
    M, N, K = 512, 640, 768
    A, B = synth.matmul_outlier(M, N, K, seed=61)
    C = host(_mm(nk, dev(A), dev(B), M, N, prec))
    R32 = O.matmul(A, B)
    err = O.rel_frobenius(C, R32)
    assert err <= TOL[prec], err
    if prec == "bf16":
        assert O.rel_frobenius(C, O.matmul_precision(A, B, "bf16")) <= 1e-5
    if prec == "fp8":   # against the dequantised E4M3 inputs the result is near FP32 exact
        assert O.rel_frobenius(C, O.matmul_precision(A, B, "fp8")) <= 1e-5


SCHEDULES = [(128, bn, 64, 1, st, sk) for bn in (64, 128, 256) for st in (2, 4) for sk in (1, 3)]
# CTA pairs issuing 2-SM MMAs (tile_m 256, cluster 2)
SCHEDULES += [(256, bn, 64, 2, st, sk) for bn in (64, 128, 256) for st in (3, 6) for sk in (1, 3)]
# wide pair tiles: 256 x 512 as two N = 256 accumulator chains
SCHEDULES += [(256, 512, 64, 2, st, sk) for st in (2, 4) for sk in (1, 3)]
# tall tiles: 2 or 4 stacked M tiles as independent chains sharing B (one CTA)
SCHEDULES += [(256, bn, 64, 1, st, sk) for bn in (64, 128) for st in (2, 4) for sk in (1, 3)]
SCHEDULES += [(512, 64, 64, 1, st, sk) for st in (2, 3) for sk in (1, 3)]


@pytest.mark.parametrize("sched", SCHEDULES)
def test_bf16_schedules_bitwise(nk, sched):
    M, N, K = 300, 520, 700
    A = synth.small_ints(62, 1, (M, K))
    B = synth.small_ints(62, 2, (K, N))
    C = host(_mm(nk, dev(A), dev(B), M, N, "bf16", schedule=sched))
    np.testing.assert_array_equal(C, O.matmul(A, B))


@pytest.mark.parametrize("sched", [(128, 64, 64, 1, 2, 1), (128, 128, 64, 1, 3, 2), (128, 64, 64, 1, 4, 3),
                                   (256, 128, 64, 2, 3, 1), (256, 64, 64, 2, 4, 2)])
def test_bf16x3_schedules_bitwise(nk, sched):
    M, N, K = 260, 200, 384
    A = synth.small_ints(67, 1, (M, K))
    B = synth.small_ints(67, 2, (K, N))
    C = host(_mm(nk, dev(A), dev(B), M, N, "bf16x3", schedule=sched))
    np.testing.assert_array_equal(C, O.matmul(A, B))


@pytest.mark.parametrize("sched", [(128, 128, 128, 1, 4, 1), (128, 256, 128, 1, 4, 2), (128, 64, 128, 1, 3, 1),
                                   (256, 256, 128, 2, 6, 1), (256, 128, 128, 2, 4, 2),
                                   (256, 512, 128, 2, 4, 1), (256, 512, 128, 2, 3, 2),
                                   (256, 128, 128, 1, 4, 1), (512, 64, 128, 1, 3, 2)])
def test_fp8_schedules_bitwise(nk, sched):
    M, N, K = 260, 384, 640
    A = synth.small_ints(63, 1, (M, K)) / 2
    B = synth.small_ints(63, 2, (K, N)) / 2
    A.flat[0], B.flat[0] = 3.5, 3.5
    C = host(_mm(nk, dev(A), dev(B), M, N, "fp8", schedule=sched))
    np.testing.assert_array_equal(C, O.matmul_precision(A, B, "fp8"))


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "fp8"])
def test_epilogue_layouts_and_transpose_identity(nk, prec):
    M, N, K = 192, 320, 256
    A, B = synth.matmul_outlier(M, N, K, seed=64)
    C0 = synth.uniform(64, 3, (M, N))
    bias = synth.uniform(64, 4, (N,), -5, 5)
    R = O.epilogue(O.matmul(A, B), c_in=C0, bias=bias, relu=True, beta=1.0)
    for a in (dev(A), colmajor(A)):
        for b in (dev(B), colmajor(B)):
            for cm in (False, True):
                c = dev(C0) if not cm else colmajor(C0)
                _mm(nk, a, b, M, N, prec, c=c, bias=dev(bias), relu=True, accumulate=True)
                assert O.rel_frobenius(host(c), R) <= TOL[prec]


def test_bf16_direct_operands(nk):
    M, N, K = 256, 384, 512
    A, B = synth.matmul_outlier(M, N, K, seed=65)
    a16 = dev(A).to(torch.bfloat16)
    bt16 = dev(np.ascontiguousarray(B.T)).to(torch.bfloat16)   # [N,K] row-major = B column-major
    C = host(_mm(nk, a16, bt16.t(), M, N, "bf16"))
    assert O.rel_frobenius(C, O.matmul_precision(A, B, "bf16")) <= 1e-5


@pytest.mark.parametrize("n", [4096, 8192])
@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
def test_full_size_sampled_rows(nk, n, prec):
    A, B = synth.matmul_outlier(n, n, n)
    C = _mm(nk, dev(A), dev(B), n, n, prec)
    rows = np.unique(synth.raw_u64(66, n, 512) % np.uint64(n)).astype(np.int64)   # ~512 sampled rows
    got = host(C[torch.from_numpy(rows).to(DEV)])
    R = O.matmul(A[rows], B)
    err = O.rel_frobenius(got, R)
    assert err <= TOL[prec], err
    if prec == "bf16":
        Rb = O.matmul(O.bf16_rn(A[rows]), O.bf16_rn(B))
        assert O.rel_frobenius(got, Rb) <= 1e-5


@pytest.mark.parametrize("prec,sched", [("bf16", (256, 256, 64, 2, 6, 1)), ("fp8", (256, 256, 128, 2, 6, 1)),
                                        ("bf16x3", (256, 128, 64, 2, 3, 1)), ("bf16", (256, 512, 64, 2, 4, 1)),
                                        ("fp8", (256, 512, 128, 2, 4, 1))])
def test_pair_full_size_sampled_rows(nk, prec, sched):
    n = 8192
    A, B = synth.matmul_outlier(n, n, n)
    C = _mm(nk, dev(A), dev(B), n, n, prec, schedule=sched)
    rows = np.unique(synth.raw_u64(68, n, 512) % np.uint64(n)).astype(np.int64)
    got = host(C[torch.from_numpy(rows).to(DEV)])
    assert O.rel_frobenius(got, O.matmul(A[rows], B)) <= TOL[prec]
    if prec == "bf16":
        assert O.rel_frobenius(got, O.matmul(O.bf16_rn(A[rows]), O.bf16_rn(B))) <= 1e-5
