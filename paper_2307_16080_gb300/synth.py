"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module only draws numbers and lays out shapes; it holds none of the
contraction arithmetic, so both the CUDA path and the FP64 oracle can be fed
from it without sharing any of the method's code.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used counter-style: output ``i`` of stream
``s`` is ``mix(s + (i + 1) * GAMMA)``.  Uniforms take the top 53 bits; normals
use the Box-Muller transform in FP64; every float tensor is rounded to FP32
with round-to-nearest-even (numpy's cast).

Workload recipes (shapes and value distributions of the dense contractions
that nelli lowers: the matmul of Listing "for->affine", the linalg.generic
matmul of Listing "linalg-matmul" and the conv of Listing "2dnchwconv",
the latter adapted to NHWC/HWCF).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 23


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, stream: int) -> np.uint64:
    """Seed of an independent stream, derived by mixing (seed, stream)."""
    with np.errstate(over="ignore"):
        z = np.array([(seed * 0x100000001B3 + stream * 0x2545F4914F6CDD1D) & (2**64 - 1)],
                     dtype=np.uint64)
        return _mix(z + GAMMA)[0]


def raw_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the SplitMix64 stream (uint64)."""
    s = stream_seed(seed, stream)
    out = np.empty(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for a in range(0, n, _CHUNK):
            b = min(n, a + _CHUNK)
            ctr = np.arange(offset + a + 1, offset + b + 1, dtype=np.uint64)
            out[a:b] = _mix(s + ctr * GAMMA)
    return out


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """FP64 uniforms in [0, 1) with 53 random bits."""
    return (raw_u64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, stream: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape))
    u = uniform01(seed, stream, n)
    return (lo + (hi - lo) * u).astype(np.float32).reshape(shape)


def normal(seed: int, stream: int, shape, sigma: float = 1.0, offset: int = 0) -> np.ndarray:
    """Box-Muller normals: z = sqrt(-2 ln(1-u1)) cos(2 pi u2), in FP64 then FP32.
    `offset` skips that many normals of the stream (element `offset` of a
    larger tensor drawn from the same stream comes first)."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float32)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        u = uniform01(seed, stream, 2 * (b - a), 2 * (offset + a))
        r = np.sqrt(-2.0 * np.log1p(-u[0::2]))
        out[a:b] = (sigma * r * np.cos(2.0 * math.pi * u[1::2])).astype(np.float32)
    return out.reshape(shape)


def half_normal(seed: int, stream: int, shape, sigma: float = 1.0) -> np.ndarray:
    return np.abs(normal(seed, stream, shape, sigma))


def outlier_normal(seed: int, stream: int, shape, p: float = 0.01,
                   factor: float = 100.0, offset: int = 0) -> np.ndarray:
    """N(0,1) with each entry independently scaled by ``factor`` with prob. ``p``
    (`offset` as for `normal`)."""
    z = normal(seed, stream, shape, offset=offset).reshape(-1)
    n = z.size
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        hit = uniform01(seed, stream + 1_000_003, b - a, offset + a) < p
        z[a:b][hit] *= np.float32(factor)
    return z.reshape(shape)


def small_ints(seed: int, stream: int, shape, lo: int = -4, hi: int = 4) -> np.ndarray:
    """Integers uniform in [lo, hi] as FP32 (exact in BF16 and E4M3 for |v| <= 16)."""
    n = int(np.prod(shape))
    r = raw_u64(seed, stream, n) % np.uint64(hi - lo + 1)
    return (r.astype(np.int64) + lo).astype(np.float32).reshape(shape)


def log_uniform_sizes(seed: int, stream: int, count: int, lo: int = 32, hi: int = 2048,
                      multiple: int = 16) -> np.ndarray:
    """round_multiple(exp(U[ln lo, ln hi])), clamped to [lo, hi]."""
    u = uniform01(seed, stream, count)
    x = np.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u)
    r = np.rint(x / multiple) * multiple
    return np.clip(r, lo, hi).astype(np.int64)


# ---------------------------------------------------------------- recipes
SEED_MATMUL_256 = 1
SEED_CONV_FP32 = 2
SEED_SWEEP = 3
SEED_GROUPED = 4
SEED_COSTMODEL = 5


def matmul_uniform(M: int, N: int, K: int, seed: int = SEED_MATMUL_256):
    """A [M,K], B [K,N] ~ U[-1,1]; C zero-initialised."""
    A = uniform(seed, 0, (M, K))
    B = uniform(seed, 1, (K, N))
    return A, B


def matmul_outlier(M: int, N: int, K: int, seed: int = SEED_SWEEP, rows=None):
    """A, B ~ N(0,1) with 1% of entries scaled by 100 (precision sweep recipe).
    rows = (r0, r1) draws only rows r0..r1-1 of the M-row A (a row block of
    the same matrix, for one rank of a row-sharded matmul)."""
    r0, r1 = (0, M) if rows is None else rows
    A = outlier_normal(seed, 10 + 2 * (M % 997), (r1 - r0, K), offset=r0 * K)
    B = outlier_normal(seed, 11 + 2 * (N % 997), (K, N))
    return A, B


def conv_resnet_block(N: int = 8, H: int = 56, W: int = 56, C: int = 64, F: int = 64,
                      KH: int = 3, KW: int = 3, seed: int = SEED_CONV_FP32):
    """I ~ |N(0,1)| [N,H,W,C]; W ~ N(0, sqrt(2/(KH*KW*C))) [KH,KW,C,F]; bias ~ U[-0.1,0.1]."""
    I = half_normal(seed, 20, (N, H, W, C))
    Wt = normal(seed, 21, (KH, KW, C, F), sigma=math.sqrt(2.0 / (KH * KW * C)))
    bias = uniform(seed, 22, (F,), -0.1, 0.1)
    return I, Wt, bias


def grouped_problems(G: int = 512, seed: int = SEED_GROUPED):
    """Shapes (M, N, K) of G independent GEMMs, each log-uniform in [32, 2048], x16."""
    M = log_uniform_sizes(seed, 30, G)
    N = log_uniform_sizes(seed, 31, G)
    K = log_uniform_sizes(seed, 32, G)
    return np.stack([M, N, K], axis=1)


def grouped_operands(shapes, seed: int = SEED_GROUPED):
    """Entries U[-1,1] for each group's A [M,K] and B [K,N]."""
    As, Bs = [], []
    for g, (M, N, K) in enumerate(shapes):
        As.append(uniform(seed, 1000 + 2 * g, (int(M), int(K))))
        Bs.append(uniform(seed, 1001 + 2 * g, (int(K), int(N))))
    return As, Bs


def resnet_stack(batch: int):
    """20-layer ResNet-style conv stack (56->7 spatial, 64->512 channels).

    Each entry: dict(N, H, W, C, F, KH, KW, stride, pad).
    56x56: 4 x (3x3 s1 64->64); then for (128@28, 256@14, 512@7): a 3x3 s2
    conv, a 1x1 s2 projection and 3 x (3x3 s1); then a 1x1 s1 512->512 @7.
    """
    layers = []
    for _ in range(4):
        layers.append(dict(N=batch, H=56, W=56, C=64, F=64, KH=3, KW=3, stride=1, pad=1))
    cin, hin = 64, 56
    for cout, hout in ((128, 28), (256, 14), (512, 7)):
        layers.append(dict(N=batch, H=hin, W=hin, C=cin, F=cout, KH=3, KW=3, stride=2, pad=1))
        layers.append(dict(N=batch, H=hin, W=hin, C=cin, F=cout, KH=1, KW=1, stride=2, pad=0))
        for _ in range(3):
            layers.append(dict(N=batch, H=hout, W=hout, C=cout, F=cout, KH=3, KW=3, stride=1, pad=1))
        cin, hin = cout, hout
    layers.append(dict(N=batch, H=7, W=7, C=512, F=512, KH=1, KW=1, stride=1, pad=0))
    assert len(layers) == 20
    return layers
