"""Multi-GPU sharding of the contractions (one process per GPU).

The path shards with no exchange step: independent problems (weak scaling),
row blocks of a matmul, images of a convolution batch, or whole groups of a
grouped GEMM.  Groups are spread by longest-processing-time first (Graham's
LPT rule) on a cost estimate, so each rank's persistent launch gets about the
same work.  Timing across ranks is the maximum of the per-rank times.  No
data-path collective is used; `torch.distributed` carries only the barrier
and the timing reduction.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_assign(costs, world: int):
    """Assign items to `world` ranks: largest cost first, each to the least
    loaded rank (ties to the lower rank).  Returns (rank of each item, load
    per rank)."""
    costs = np.asarray(costs, dtype=np.float64)
    order = np.argsort(-costs, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    owner = np.empty(len(costs), dtype=np.int64)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + float(costs[i]), r))
    loads = np.zeros(world)
    np.add.at(loads, owner, costs)
    return owner, loads


def gemm_flops(shapes):
    """2*M*N*K per group -- the cost estimate used for grouped sharding."""
    s = np.asarray(shapes, dtype=np.float64)
    return 2.0 * s[:, 0] * s[:, 1] * s[:, 2]


def row_blocks(M: int, world: int, align: int = 128):
    """Contiguous row ranges [r0, r1) of an M-row matmul, one per rank, cut on
    `align`-row boundaries (whole output tiles)."""
    tiles = (M + align - 1) // align
    base, extra = divmod(tiles, world)
    out, t = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((min(M, t * align), min(M, (t + n) * align)))
        t += n
    return out


def max_over_ranks(value: float, group=None) -> float:
    """The largest `value` over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
