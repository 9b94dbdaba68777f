"""Host logic of the multi-GPU path, on CPU: LPT group assignment, row and
batch blocks, the max-over-ranks timing reduction, and the whole split ->
per-rank compute -> assembly path with two gloo ranks.  Each rank computes
its shard with a host stand-in (the FP64 oracle) in place of the GPU call,
so what is checked is the partition and the reassembly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2307_16080_gb300 import shard, synth


def test_lpt_balances_the_grouped_config():
    shapes = synth.grouped_problems(512)
    cost = shard.gemm_flops(shapes)
    for world in (2, 4, 8):
        owner, loads = shard.lpt_assign(cost, world)
        assert set(owner.tolist()) == set(range(world))
        assert abs(loads.sum() - cost.sum()) <= 1e-9 * cost.sum()
        # Graham's bound for LPT: makespan <= (4/3 - 1/(3m)) * optimum, and optimum >= mean
        assert loads.max() <= (4 / 3 - 1 / (3 * world)) * max(loads.mean(), cost.max()) + 1e-6
        assert loads.max() / loads.mean() < 1.01     # 512 items spread this evenly


def test_lpt_small_exact_case():
    owner, loads = shard.lpt_assign([7, 5, 4, 3, 1], 2)
    assert sorted(loads.tolist()) == [10.0, 10.0]


def test_row_blocks_cover_once():
    for M, world in ((8192, 8), (1000, 3), (100, 4), (129, 2)):
        blocks = shard.row_blocks(M, world)
        assert blocks[0][0] == 0 and blocks[-1][1] == M
        for (a, b), (c, d) in zip(blocks, blocks[1:]):
            assert b == c and a <= b
        assert all((a % 128 == 0) for a, _ in blocks if a < M)


def test_batch_blocks_cover_once():
    for N, world in ((32, 8), (8, 3), (1, 2), (7, 7)):
        blocks = shard.batch_blocks(N, world)
        assert blocks[0][0] == 0 and blocks[-1][1] == N
        sizes = [b - a for a, b in blocks]
        assert max(sizes) - min(sizes) <= 1
        for (a, b), (c, d) in zip(blocks, blocks[1:]):
            assert b == c


def test_row_block_inputs_are_rows_of_the_whole_matrix():
    """A rank draws only its row block of A; it equals those rows of the
    matrix drawn whole, so the sharded problem is the same problem."""
    M, N, K = 640, 48, 96
    A, B = synth.matmul_outlier(M, N, K)
    for r0, r1 in shard.row_blocks(M, 3):
        Ar, Br = synth.matmul_outlier(M, N, K, rows=(r0, r1))
        np.testing.assert_array_equal(Ar, A[r0:r1])
        np.testing.assert_array_equal(Br, B)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _timing_worker(rank, world, port, out):
    dist = _init(rank, world, port)
    shapes = synth.grouped_problems(64)
    owner, _ = shard.lpt_assign(shard.gemm_flops(shapes), world)
    mine = float(shard.gemm_flops(shapes)[owner == rank].sum())
    out[rank] = (shard.max_over_ranks(mine), mine)
    dist.barrier()
    dist.destroy_process_group()


def _split_worker(rank, world, port, out):
    """One rank of the sharded path: its row block of the matmul, its LPT
    groups of a grouped GEMM, its images of a convolution -- each computed
    by the host stand-in -- then gathered in rank order."""
    import oracle.nk_oracle as O
    dist = _init(rank, world, port)
    res = {}
    # matmul: row blocks of A, B replicated
    M, N, K = 700, 96, 160
    blocks = shard.row_blocks(M, world)
    r0, r1 = blocks[rank]
    A, B = synth.matmul_outlier(M, N, K, rows=(r0, r1))
    parts = shard.gather_shards(O.matmul(A, B))
    res["matmul"] = shard.assemble_blocks(blocks, parts)
    # grouped: whole groups by LPT on 2*M*N*K
    shapes = synth.grouped_problems(24)
    As, Bs = synth.grouped_operands(shapes)
    owner, _ = shard.lpt_assign(shard.gemm_flops(shapes), world)
    mine = shard.groups_of_rank(owner, rank)
    flat = np.concatenate([O.matmul(As[g], Bs[g]).ravel() for g in mine]) if len(mine) else np.zeros(0)
    res["grouped_parts"] = [p for p in shard.gather_shards(flat)]
    res["grouped_owner"] = owner
    # conv: images of the batch
    I, W, bias = synth.conv_resnet_block(N=5, H=12, W=12, C=16, F=8)
    bb = shard.batch_blocks(5, world)
    n0, n1 = bb[rank]
    o = O.epilogue(O.conv2d_nhwc_hwcf(I[n0:n1], W, pad=(1, 1, 1, 1)), bias=bias, relu=True)
    res["conv"] = shard.assemble_blocks(bb, shard.gather_shards(o))
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def _run(target, world=2):
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=target, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    return dict(out)


def test_max_over_ranks_two_gloo_ranks():
    out = _run(_timing_worker)
    mx = max(v[1] for v in out.values())
    assert all(v[0] == mx for v in out.values())
    assert abs(sum(v[1] for v in out.values()) - shard.gemm_flops(synth.grouped_problems(64)).sum()) < 1


@pytest.mark.timeout(300)
def test_sharded_results_assemble_to_the_whole_problem():
    import oracle.nk_oracle as O
    out = _run(_split_worker)
    # every rank holds the same assembled results
    for key in ("matmul", "conv"):
        np.testing.assert_array_equal(out[0][key], out[1][key])
    M, N, K = 700, 96, 160
    A, B = synth.matmul_outlier(M, N, K)
    np.testing.assert_array_equal(out[0]["matmul"], O.matmul(A, B))
    I, W, bias = synth.conv_resnet_block(N=5, H=12, W=12, C=16, F=8)
    ref = O.epilogue(O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)), bias=bias, relu=True)
    np.testing.assert_array_equal(out[0]["conv"], ref)
    shapes = synth.grouped_problems(24)
    As, Bs = synth.grouped_operands(shapes)
    owner = out[0]["grouped_owner"]
    parts = out[0]["grouped_parts"]
    for rank in range(2):
        mine = shard.groups_of_rank(owner, rank)
        off = 0
        for g in mine:
            ref = O.matmul(As[g], Bs[g])
            np.testing.assert_array_equal(parts[rank][off:off + ref.size].reshape(ref.shape), ref)
            off += ref.size
        assert off == parts[rank].size
    assert sorted(np.concatenate([shard.groups_of_rank(owner, r) for r in range(2)]).tolist()) == list(range(24))
