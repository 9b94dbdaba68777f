"""Brute force on tiny shapes: every (M, N, K) with M, N, K in
{1..8, 15, 16, 17, 31, 33, 127, 129} (3375 shapes) through nk_matmul in
each precision, bitwise against the FP64 oracle.

Entries are small integers in [-4, 4]: every product and partial sum is an
integer below 2^24, exact in FP32 accumulation whatever the order, and the
inputs are exact in BF16 (hi = x, lo = 0 for BF16x3) and, with scale 1, in
E4M3 (passed already quantised).  So any difference is a kernel error:
a dropped tile edge, a wrong stride, a lost K remainder.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import DEV

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 4, 5, 6, 7, 8, 15, 16, 17, 31, 33, 127, 129]


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def operands():
    """One [129, 129] A and B of small integers; each shape takes a corner."""
    A = synth.small_ints(161, 1, (129, 129))
    B = synth.small_ints(161, 2, (129, 129))
    return A, B


def _e4m3_rows(x, ld):
    """Device E4M3 [rows, cols] view of x, rows padded to `ld` bytes (a
    16-byte multiple, as TMA needs)."""
    rows, cols = x.shape
    buf = torch.zeros(rows, ld, dtype=torch.float8_e4m3fn, device=DEV)
    buf[:, :cols] = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(DEV).to(torch.float8_e4m3fn)
    return buf[:, :cols]


@pytest.mark.parametrize("prec", ["f32", "bf16", "bf16x3", "fp8"])
def test_every_tiny_shape_bitwise(nk, operands, prec):
    A, B = operands
    bad = []
    for M, N, K in itertools.product(SIZES, SIZES, SIZES):
        a, b = A[:M, :K], B[:K, :N]
        c = torch.full((M, N), float("nan"), device=DEV)
        if prec == "fp8":
            ld = (K + 15) // 16 * 16
            a8 = _e4m3_rows(a, ld)
            bt8 = _e4m3_rows(np.ascontiguousarray(b.T), ld)
            nk.nk_matmul(a8, bt8.t(), c, precision="fp8", scale_a=1.0, scale_b=1.0)
        else:
            nk.nk_matmul(torch.from_numpy(np.ascontiguousarray(a)).to(DEV),
                         torch.from_numpy(np.ascontiguousarray(b)).to(DEV), c, precision=prec)
        got = c.cpu().numpy()
        if not np.array_equal(got, O.matmul(a, b)):
            bad.append((M, N, K))
    nk.nk_sync_status()
    assert not bad, f"{len(bad)} shapes differ, first {bad[:5]}"
