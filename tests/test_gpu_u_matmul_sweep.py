"""Seeded sweep of random nk_matmul calls, bitwise against the oracle, with
every output inside a canary-filled buffer.

Each case draws a precision, M, N, K in [1, 700], the major-ness of A, B
and C and whether their leading dimensions are padded, bias / ReLU /
accumulate, and either the built-in schedule or a random legal one
(nk_enumerate_schedules for the tensor-core precisions, SIMT tiles with
split-K for FP32).  Entries are small integers (half-integers with amax
3.5 for E4M3: scale 128, exact codes), so every result is exact; C's
padding and everything around it must keep its sentinels.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from paper_2307_16080_gb300 import nk_tune as nt
from tests.gpu_util import DEV, Canary

pytestmark = pytest.mark.gpu

NCASES = 96
PRECS = ["f32", "bf16", "bf16x3", "fp8"]


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


def _operand(x, col_major, pad):
    """Device FP32 tensor with x's values: row- or column-major, leading
    dimension padded by `pad` elements."""
    r, c = x.shape
    if col_major:
        buf = torch.zeros(c, r + pad, device=DEV)
        buf[:, :r] = torch.from_numpy(np.ascontiguousarray(x.T)).to(DEV)
        return buf[:, :r].t()
    buf = torch.zeros(r, c + pad, device=DEV)
    buf[:, :c] = torch.from_numpy(x).to(DEV)
    return buf[:, :c]


@pytest.mark.parametrize("case", range(NCASES))
def test_random_matmul_bitwise(nk, case):
    u = synth.uniform01(191, case, 16)
    prec = PRECS[case % 4]
    M, N, K = (1 + int(u[0] ** 2 * 700), 1 + int(u[1] ** 2 * 700), 1 + int(u[2] ** 2 * 700))
    A = synth.small_ints(192, 2 * case, (M, K))
    B = synth.small_ints(192, 2 * case + 1, (K, N))
    if prec == "fp8":
        A, B = A / 2, B / 2
        A.flat[0], B.flat[0] = 3.5, -3.5
    a_col, b_col, c_col = u[3] < 0.3, u[4] < 0.3, u[5] < 0.25
    pads = [int(u[6] * 3) * 4, int(u[7] * 3) * 4, [0, 1, 4, 13][int(u[8] * 4)]]
    bias = synth.small_ints(193, case, (N,)) if u[9] < 0.5 else None
    relu = bool(u[10] < 0.4)
    acc = bool(u[11] < 0.3)
    sched = None
    if u[12] < 0.7 and not c_col:   # a column-major C runs as C^T = B^T A^T: keep its built-in schedule
        if prec == "f32":
            sched = [(64, 64, 16, 1, 2, 1), (64, 64, 16, 1, 2, 3), (128, 64, 16, 1, 2, 2)][int(u[13] * 3)]
        else:
            cands = nt.nk_enumerate_schedules(nt.matmul_problem(M, N, K, prec))
            sched = cands[int(u[13] * len(cands))] if cands else None
    ldc = (M if c_col else N) + pads[2]
    c = Canary((M, N), strides=(1, ldc) if c_col else (ldc, 1))
    C0 = synth.small_ints(194, case, (M, N))
    if acc:
        c.t.copy_(torch.from_numpy(C0).to(DEV))
    nk.nk_matmul(_operand(A, a_col, pads[0]), _operand(B, b_col, pads[1]), c.t, precision=prec, schedule=sched,
                 bias=torch.from_numpy(bias).to(DEV) if bias is not None else None, relu=relu, accumulate=acc)
    nk.nk_sync_status()
    c.check()
    R = O.epilogue(O.matmul_precision(A, B, prec), c_in=C0 if acc else None, bias=bias, relu=relu,
                   beta=1.0 if acc else 0.0)
    np.testing.assert_array_equal(c.t.cpu().numpy(), R, err_msg=str((prec, M, N, K, a_col, b_col, c_col, pads,
                                                                      bias is not None, relu, acc, sched)))
