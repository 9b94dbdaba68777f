"""GPU parity of the grouped persistent GEMM (uneven BF16 groups in one
launch, replayed from a CUDA graph) against the FP64 oracle."""
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


def _operands(shapes, seed, ints=False):
    As, Bs = [], []
    for g, (M, N, K) in enumerate(shapes):
        if ints:
            As.append(synth.small_ints(seed, 2 * g, (M, K)))
            Bs.append(synth.small_ints(seed, 2 * g + 1, (K, N)))
        else:
            As.append(synth.uniform(seed, 1000 + 2 * g, (M, K)))
            Bs.append(synth.uniform(seed, 1001 + 2 * g, (K, N)))
    a = [dev(x).to(torch.bfloat16) for x in As]
    bt = [dev(np.ascontiguousarray(x.T)).to(torch.bfloat16) for x in Bs]
    c = [torch.empty(M, N, device=DEV) for (M, N, K) in shapes]
    return As, Bs, a, bt, c


SMALL = [(33, 17, 16), (128, 256, 64), (200, 130, 520), (16, 16, 16), (300, 64, 2048), (129, 511, 80),
         (1, 1, 8), (256, 384, 1024)]


@pytest.mark.parametrize("tile_m,cluster", [(128, 1), (256, 2)])
@pytest.mark.parametrize("tile_n", [64, 128, 256])
def test_grouped_small_ints_bitwise(nk, tile_n, tile_m, cluster):
    """One CTA per 128-row tile, or a CTA pair per 256-row tile (cta_group::2,
    half of B in each CTA); groups smaller than a tile included."""
    As, Bs, a, bt, c = _operands(SMALL, 70, ints=True)
    groups, G = nk.make_groups(a, bt, c)
    plan = nk.nk_grouped_plan_create(groups, G, schedule=(tile_m, tile_n, 0, cluster, 0, 0))
    nk.nk_grouped_plan_run(plan)
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)
    for g in range(G):
        np.testing.assert_array_equal(host(c[g]), O.matmul(As[g], Bs[g]))


def test_grouped_512_config_graph_replay(nk):
    shapes = [tuple(int(v) for v in s) for s in synth.grouped_problems(512)]
    As, Bs, a, bt, c = _operands(shapes, synth.SEED_GROUPED)
    groups, G = nk.make_groups(a, bt, c)
    plan = nk.nk_grouped_plan_create(groups, G)
    nk.nk_grouped_plan_run(plan)
    nk.nk_sync_status()
    eager = [host(x).copy() for x in c]
    worst32, worst16 = 0.0, 0.0
    for g in range(G):
        worst32 = max(worst32, O.rel_frobenius(eager[g], O.matmul(As[g], Bs[g])))
        worst16 = max(worst16, O.rel_frobenius(eager[g], O.matmul_precision(As[g], Bs[g], "bf16")))
    assert worst16 <= 1e-5 and worst32 <= 8e-3, (worst16, worst32)
    for x in c:
        x.zero_()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            nk.nk_grouped_plan_run(plan)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        for x in c:
            x.fill_(7.0)
        graph.replay()
        torch.cuda.synchronize()
        for g in range(G):
            np.testing.assert_array_equal(host(c[g]), eager[g])
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)


def test_one_shot_matches_plan_and_accumulate(nk):
    shapes = [(64, 96, 48), (300, 200, 256), (17, 33, 16)]
    As, Bs, a, bt, c = _operands(shapes, 71)
    C0 = [synth.uniform(71, 50 + g, (M, N)) for g, (M, N, K) in enumerate(shapes)]
    for g in range(len(c)):
        c[g].copy_(dev(C0[g]))
    groups, G = nk.make_groups(a, bt, c, accumulate=True)
    nk.nk_batch_matmul_grouped(groups, G)
    nk.nk_sync_status()
    for g in range(G):
        R = O.epilogue(O.matmul_precision(As[g], Bs[g], "bf16"), c_in=C0[g], beta=1.0)
        assert O.rel_frobenius(host(c[g]), R) <= 1e-5


def test_single_group_equals_matmul(nk):
    M, N, K = 384, 256, 1024
    As, Bs, a, bt, c = _operands([(M, N, K)], 72)
    groups, G = nk.make_groups(a, bt, c)
    plan = nk.nk_grouped_plan_create(groups, G, schedule=(128, 128, 64, 1, 4, 1))
    nk.nk_grouped_plan_run(plan)
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)
    ref = torch.empty(M, N, device=DEV)
    nk.nk_matmul(a[0], bt[0].t(), ref, precision="bf16", schedule=(128, 128, 64, 1, 4, 1))
    nk.nk_sync_status()
    np.testing.assert_array_equal(host(c[0]), host(ref))


def test_uniform_batch_is_batch_matmul(nk):
    Bn, M, N, K = 6, 128, 192, 320
    A = synth.uniform(73, 0, (Bn, M, K))
    B = synth.uniform(73, 1, (Bn, K, N))
    a = dev(A).to(torch.bfloat16)
    bt = dev(np.ascontiguousarray(B.transpose(0, 2, 1))).to(torch.bfloat16)
    c = torch.empty(Bn, M, N, device=DEV)
    groups, G = nk.make_groups(list(a), list(bt), list(c))
    nk.nk_batch_matmul_grouped(groups, G)
    nk.nk_sync_status()
    R = O.batch_matmul(O.bf16_rn(A), O.bf16_rn(B))
    assert O.rel_frobenius(host(c), R) <= 1e-5


def test_grouped_rejects_bad_groups(nk):
    a = torch.empty(32, 10, dtype=torch.bfloat16, device=DEV)    # row of 20 bytes: not TMA-legal
    bt = torch.empty(16, 10, dtype=torch.bfloat16, device=DEV)
    c = torch.empty(32, 16, device=DEV)
    groups, G = nk.make_groups([a], [bt], [c])
    with pytest.raises(nk.NkError) as e:
        nk.nk_batch_matmul_grouped(groups, G)
    assert e.value.status == -3


def test_grouped_tune_picks_a_legal_fast_schedule_and_stays_exact(nk):
    """nk_grouped_tune times every legal grouped schedule on the caller's
    groups; the winner is no slower than the built-in choice (it is one of
    the candidates) and a plan built with it is still exact."""
    from paper_2307_16080_gb300 import nk_tune as nt
    As, Bs, a, bt, c = _operands(SMALL, 71, ints=True)
    groups, G = nk.make_groups(a, bt, c, accumulate=True)   # accumulate is ignored while tuning
    best, rep = nt.nk_grouped_tune(groups, G, reps=3)
    assert rep.timed == rep.candidates >= 10
    assert (best[0], best[3]) in ((128, 1), (256, 2)) and best[1] in (64, 128, 256) and best[5] == 1
    assert 2 <= best[4] <= 8
    assert 0 < rep.best_ms <= rep.default_ms * 1.05
    groups, G = nk.make_groups(a, bt, c)
    plan = nk.nk_grouped_plan_create(groups, G, schedule=best)
    nk.nk_grouped_plan_run(plan)
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)
    for g in range(G):
        np.testing.assert_array_equal(host(c[g]), O.matmul(As[g], Bs[g]))


def test_grouped_512_pair_tiles(nk):
    """The 512-group config on CTA pairs (256 x 256 tiles), graph-replayed,
    within the BF16 tolerances on every group."""
    shapes = [tuple(int(v) for v in s) for s in synth.grouped_problems(512)]
    As, Bs, a, bt, c = _operands(shapes, synth.SEED_GROUPED)
    groups, G = nk.make_groups(a, bt, c)
    plan = nk.nk_grouped_plan_create(groups, G, schedule=(256, 256, 64, 2, 4, 1))
    nk.nk_grouped_plan_run(plan)
    nk.nk_sync_status()
    nk.nk_grouped_plan_destroy(plan)
    for g in range(0, G, 7):
        got = host(c[g])
        assert O.rel_frobenius(got, O.matmul(O.bf16_rn(As[g]), O.bf16_rn(Bs[g]))) <= 1e-5, g
        assert O.rel_frobenius(got, O.matmul(As[g], Bs[g])) <= 8e-3, g
