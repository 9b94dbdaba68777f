"""Degenerate and edge cases through the C ABI: empty extents, an empty
reduction (K = 0, where the contraction is the zero-filled output of
Listing "listing1" and only the epilogue remains), single rows / columns,
and non-finite inputs."""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import DEV, dev, host

pytestmark = pytest.mark.gpu
PRECS = ["f32", "bf16", "bf16x3", "fp8"]


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("M,N", [(0, 5), (4, 0), (0, 0)])
def test_empty_output_is_a_no_op(nk, prec, M, N):
    a = torch.zeros(M, 8, device=DEV)
    b = torch.zeros(8, N, device=DEV)
    c = torch.full((M, N), 7.0, device=DEV)
    nk.nk_matmul(a, b, c, precision=prec)
    nk.nk_sync_status()
    assert c.numel() == 0 or bool(torch.all(c == 7.0))


@pytest.mark.parametrize("prec", PRECS)
def test_empty_reduction_leaves_the_epilogue(nk, prec):
    M, N = 37, 70
    a = torch.zeros(M, 0, device=DEV)
    b = torch.zeros(0, N, device=DEV)
    C0 = synth.uniform(100, 0, (M, N))
    bias = synth.uniform(100, 1, (N,), -1, 1)
    c = dev(C0)
    nk.nk_matmul(a, b, c, precision=prec, bias=dev(bias), relu=True, accumulate=True)
    nk.nk_sync_status()
    R = O.epilogue(np.zeros((M, N)), c_in=C0, bias=bias, relu=True, beta=1.0)
    np.testing.assert_allclose(host(c), R, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("M,N,K", [(1, 300, 40), (300, 1, 40), (1, 1, 4096), (2, 3, 1)])
def test_single_rows_and_columns(nk, prec, M, N, K):
    A = synth.small_ints(101, M * 7 + N, (M, K))
    B = synth.small_ints(101, N * 5 + K, (K, N))
    if prec == "fp8":
        A, B = A / 2, B / 2
        A.flat[0], B.flat[0] = 3.5, 3.5
    c = torch.empty(M, N, device=DEV)
    nk.nk_matmul(dev(A), dev(B), c, precision=prec)
    nk.nk_sync_status()
    np.testing.assert_array_equal(host(c), O.matmul_precision(A, B, prec))


def test_nan_and_inf_propagate_f32_and_bf16(nk):
    A = synth.uniform(102, 0, (64, 96))
    B = synth.uniform(102, 1, (96, 80))
    A[3, 5] = np.nan
    A[10, 7] = np.inf
    for prec in ("f32", "bf16"):
        c = torch.empty(64, 80, device=DEV)
        nk.nk_matmul(dev(A), dev(B), c, precision=prec, relu=True)
        nk.nk_sync_status()
        got = host(c)
        assert np.all(np.isnan(got[3])), prec                 # NaN row survives ReLU
        assert np.all(np.isinf(got[10]) | np.isnan(got[10]) | (got[10] == 0)), prec
        assert np.all(np.isfinite(np.delete(got, [3, 10], axis=0))), prec


def test_fp8_nan_input_falls_back_to_unit_scale(nk):
    A = synth.uniform(103, 0, (32, 64))
    A[0, 0] = np.nan
    amax = torch.empty(1, device=DEV)
    nk.nk_amax(dev(A), amax)
    q = torch.empty(32, 64, dtype=torch.uint8, device=DEV)
    s = torch.empty(1, device=DEV)
    nk.nk_cast_fp8(dev(A), amax, q, scale_out=s)
    torch.cuda.synchronize()
    assert np.isnan(amax.item()) and s.item() == 1.0


def test_conv_degenerate_shapes(nk):
    # 1x1 output from a full-size 3x3 window; a batch of one pixel; stride larger than the filter
    for (N, H, W, C, F, k, st, pad) in [(2, 3, 3, 8, 16, 3, (1, 1), (0, 0, 0, 0)),
                                        (1, 1, 1, 64, 64, 1, (1, 1), (0, 0, 0, 0)),
                                        (3, 10, 10, 16, 8, 1, (3, 3), (0, 0, 0, 0))]:
        I = synth.small_ints(104, H * C, (N, H, W, C))
        Wt = synth.small_ints(104, F * k, (k, k, C, F))
        R = O.conv2d_nhwc_hwcf(I, Wt, st, (1, 1), pad)
        for prec in ("f32", "bf16"):
            out = torch.empty(*R.shape, device=DEV)
            nk.nk_conv2d_nhwc_hwcf(dev(I), dev(Wt), out, stride=st, pad=pad, precision=prec)
            nk.nk_sync_status()
            np.testing.assert_array_equal(host(out), R)
