"""Multi-GPU sharding of the contractions (one process per GPU).

The only parallelism the paper uses is the output-parallel loop of the
convolution (Sec. 4.1, the scf.parallel that its GPU and OpenMP lowerings
map onto threads): every output block is independent.  Across GPUs that
gives three splits with no exchange step:

* matmul: contiguous row blocks of A (whole 128-row output tiles) with B
  replicated; rank r computes C[r0:r1, :] = A[r0:r1, :] @ B;
* grouped GEMM: whole groups, spread by longest-processing-time first
  (Graham's LPT rule) on a cost estimate, so each rank's persistent launch
  gets about the same work;
* convolution: contiguous blocks of images of the batch (every image's
  output depends on that image alone).

Each rank computes on its own device memory only.  Timing across ranks is
the maximum of the per-rank times; `assemble` gathers the shards where a
caller wants the whole result on every rank (the one collective, outside
the timed path).
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
    """2*M*N*K per group -- a cost estimate for grouped sharding when no
    measured or predicted times are at hand."""
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


def batch_blocks(N: int, world: int):
    """Contiguous image ranges [n0, n1) of a convolution batch, one per rank
    (sizes differ by at most one image)."""
    base, extra = divmod(N, world)
    out, t = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((t, t + n))
        t += n
    return out


def groups_of_rank(owner, rank: int):
    """Indices of the groups rank `rank` computes, in their original order."""
    return np.flatnonzero(np.asarray(owner) == rank)


def assemble_blocks(blocks, parts, axis: int = 0):
    """Concatenate per-rank shards (in rank order) along `axis`, checking
    that each shard has the extent its block says."""
    for (a, b), p in zip(blocks, parts):
        assert p.shape[axis] == b - a, (a, b, p.shape)
    return np.concatenate(list(parts), axis=axis)


def gather_shards(local: np.ndarray, group=None):
    """All ranks' shards of `local` (FP32/FP64 numpy arrays, first dimensions
    may differ between ranks) in rank order, on every rank."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return [local]
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    n = torch.tensor([local.shape[0]], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    rows = max(int(s.item()) for s in sizes)
    pad = np.zeros((rows,) + local.shape[1:], dtype=local.dtype)
    pad[:local.shape[0]] = local
    t = torch.from_numpy(pad).to(dev)
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    return [o.cpu().numpy()[:int(s.item())] for o, s in zip(out, sizes)]


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
