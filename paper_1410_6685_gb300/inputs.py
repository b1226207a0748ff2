"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the oracle checks and ``bench.py``.  It
holds no arithmetic of the method itself -- only random draws and the
construction of the workloads (the paper's Sec. 6 benchmarks: vector
addition, sorting, matrix multiplication, Gaussian elimination, plus the
batched-collections workload).  It imports nothing from the library's
compiled code, so importing it never loads CUDA.

Every generator is ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import numpy as np

SEED_VADD = 0
SEED_SORT_UNIFORM = 1
SEED_SORT_DISTINCT_VALUES = 2
SEED_SORT_DISTINCT_KEYS = 3
SEED_MM_A = 4
SEED_MM_B = 5
SEED_FREIVALDS = 6
SEED_GEPP = 7
SEED_BATCH_LENGTHS = 8
SEED_BATCH_DATA = 9


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_pm1(g: np.random.Generator, n: int) -> np.ndarray:
    """n binary32 values, uniform on [-1, 1)."""
    u = g.random(n, dtype=np.float32)
    return (u * np.float32(2.0) - np.float32(1.0)).astype(np.float32)


def vadd_inputs(n: int, seed: int = SEED_VADD):
    """Vector addition workload: a then b, both U[-1,1) binary32, one stream."""
    g = rng(seed)
    a = uniform_pm1(g, n)
    b = uniform_pm1(g, n)
    return a, b


def sort_keys_uniform(n: int, seed: int = SEED_SORT_UNIFORM) -> np.ndarray:
    """int32 keys uniform over the full signed range [-2^31, 2^31)."""
    g = rng(seed)
    return g.integers(-2**31, 2**31, size=n, dtype=np.int64).astype(np.int32)


def sort_keys_distinct(n: int, ndistinct: int = 256,
                       seed_values: int = SEED_SORT_DISTINCT_VALUES,
                       seed_keys: int = SEED_SORT_DISTINCT_KEYS) -> np.ndarray:
    """int32 keys drawn uniformly from `ndistinct` values, themselves uniform
    over the full int32 range."""
    values = rng(seed_values).integers(-2**31, 2**31, size=ndistinct,
                                       dtype=np.int64).astype(np.int32)
    idx = rng(seed_keys).integers(0, ndistinct, size=n, dtype=np.int64)
    return values[idx]


def matmul_inputs(n: int, seed_a: int = SEED_MM_A, seed_b: int = SEED_MM_B):
    """Square A, B with N(0,1) binary32 entries, row-major."""
    A = rng(seed_a).standard_normal((n, n), dtype=np.float32)
    B = rng(seed_b).standard_normal((n, n), dtype=np.float32)
    return A, B


def gepp_inputs(n: int, seed: int = SEED_GEPP):
    """Diagonally dominant system: off-diagonal N(0,1) binary32; a_ii = (sum of
    |a_ij|, j != i, in binary64) + 1 rounded to binary32; b = A*ones in
    binary64 from the binary32 A (so the solution is all ones)."""
    A = rng(seed).standard_normal((n, n), dtype=np.float32)
    A64 = A.astype(np.float64)
    np.fill_diagonal(A64, 0.0)
    diag = np.abs(A64).sum(axis=1) + 1.0
    np.fill_diagonal(A, diag.astype(np.float32))
    b = A.astype(np.float64).sum(axis=1)
    return A, b


def batch_lengths(nseg: int = 10000, seed: int = SEED_BATCH_LENGTHS,
                  lo_log2: int = 6, hi_log2: int = 20) -> np.ndarray:
    """Segment lengths floor(2^(lo + (hi-lo) u)), u ~ U[0,1), clamped."""
    u = rng(seed).random(nseg)
    L = np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)
    return np.clip(L, 2 ** lo_log2, 2 ** hi_log2)


def batch_offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def batch_data(total: int, seed: int = SEED_BATCH_DATA) -> np.ndarray:
    """The concatenated segments: U[-1,1) binary32."""
    return uniform_pm1(rng(seed), total)


def mlp_init(d_in: int, H: int = 64, seed: int = 11) -> np.ndarray:
    """He-style initial parameters of the 2x64 MLP in the flat layout
    [W1 (H x d_in), b1, W2 (H x H), b2, W3 (H), b3]."""
    g = rng(seed)
    W1 = g.standard_normal((H, d_in)) * np.sqrt(2.0 / d_in)
    W2 = g.standard_normal((H, H)) * np.sqrt(2.0 / H)
    W3 = g.standard_normal(H) * np.sqrt(1.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H),
                           W3, np.zeros(1)])
