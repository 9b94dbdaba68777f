"""Seeded sweep of random grouped GEMMs through plans, bitwise against the
oracle, with canary padding around every output.

Each set draws 1-40 groups with M, N in [1, 300] and K a multiple of 8 in
[8, 512] (BF16 rows of 16 bytes); the C row stride is either N (not always
a 16-byte multiple: per-lane stores) or N rounded up to 4 (16-byte rows:
the per-group TMA-store epilogue, clipped at each group's edges).  Every
set runs with the default tile, 128 x 64, 128 x 256 with four stages (one
CTA per SM, eight epilogue warps) and 256 x 128 on CTA pairs.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import Canary

pytestmark = pytest.mark.gpu

NSETS = 24
SCHEDULES = [None, (128, 64, 0, 1, 0, 0), (128, 256, 64, 1, 4, 0), (256, 128, 0, 2, 0, 0)]


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


def _group_set(i):
    u = synth.uniform01(181, i, 1 + 3 * 40)
    G = 1 + int(u[0] * 40)
    shapes = []
    for g in range(G):
        r = u[1 + 3 * g: 4 + 3 * g]
        M = 1 + int(r[0] ** 2 * 300)
        N = 1 + int(r[1] ** 2 * 300)
        K = 8 * (1 + int(r[2] * 64))
        shapes.append((M, N, K))
    aligned = i % 2 == 1   # odd sets: every C row a 16-byte multiple
    return shapes, aligned


@pytest.mark.parametrize("i", range(NSETS))
def test_random_group_sets_bitwise(nk, i):
    shapes, aligned = _group_set(i)
    As = [synth.small_ints(182 + i, 2 * g, (M, K)) for g, (M, N, K) in enumerate(shapes)]
    Bs = [synth.small_ints(182 + i, 2 * g + 1, (K, N)) for g, (M, N, K) in enumerate(shapes)]
    a16 = [torch.from_numpy(a).cuda().to(torch.bfloat16) for a in As]
    bt16 = [torch.from_numpy(np.ascontiguousarray(b.T)).cuda().to(torch.bfloat16) for b in Bs]
    for sched in SCHEDULES:
        cans = [Canary((M, N), strides=((N + 3) // 4 * 4 if aligned else N, 1)) for (M, N, K) in shapes]
        groups, G = nk.make_groups(a16, bt16, [c.t for c in cans])
        plan = nk.nk_grouped_plan_create(groups, G, schedule=sched)
        nk.nk_grouped_plan_run(plan)
        nk.nk_sync_status()
        nk.nk_grouped_plan_destroy(plan)
        for g, c in enumerate(cans):
            c.check()
            got = c.t.cpu().numpy()
            assert np.array_equal(got, O.matmul(As[g], Bs[g])), (i, sched, g, shapes[g])
