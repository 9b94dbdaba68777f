"""Host logic of the multi-GPU path, on CPU: LPT group assignment, row
blocks, and the max-over-ranks timing reduction with two gloo ranks."""
import os
import socket

import numpy as np
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


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shapes = synth.grouped_problems(64)
    owner, _ = shard.lpt_assign(shard.gemm_flops(shapes), world)
    mine = float(shard.gemm_flops(shapes)[owner == rank].sum())
    out[rank] = (shard.max_over_ranks(mine), mine)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    mx = max(v[1] for v in out.values())
    assert all(v[0] == mx for v in out.values())
    assert abs(sum(v[1] for v in out.values()) - shard.gemm_flops(synth.grouped_problems(64)).sum()) < 1
