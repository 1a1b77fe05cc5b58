"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no tropical arithmetic: it only turns (seed, stream tag,
element index) into numbers.  Both the CPU oracle and the CUDA path are fed
the arrays it returns, so neither side generates its own inputs.

Hash: the SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to a counter,
    h(seed, tag, idx) = mix64(seed * G + (tag << 40) + idx + 1),
with G the 64-bit golden-ratio increment.  Counter-based, so any element of
any matrix can be regenerated alone and generation is chunked by rows.

Shapes and distributions follow the paper's workload (random weighted
directed graphs as adjacency matrices, Sec. IV, Table II) at the sizes the
benchmark configurations name.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 0x170104733

INF_I32 = 0x3FFFFFFF       # "no edge" in int32 adjacency matrices
INF_U16 = 0x7FFF           # "no edge" in the 16-bit encoding

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def hash64(seed: int, tag: int, idx: np.ndarray) -> np.ndarray:
    """64-bit hash of element indices `idx` (uint64 array) in stream (seed, tag)."""
    base = ((seed * 0x9E3779B97F4A7C15) + ((tag & 0xFFFFFF) << 40) + 1) & 0xFFFFFFFFFFFFFFFF
    with np.errstate(over="ignore"):
        return _mix64(idx.astype(np.uint64) + np.uint64(base))


def _rows(total: int):
    start = 0
    while start < total:
        stop = min(total, start + _CHUNK)
        yield start, stop
        start = stop


def uniform_int(seed: int, tag: int, shape, lo: int, hi: int, dtype=np.int32) -> np.ndarray:
    """Integers uniform in [lo, hi] (multiply-shift range reduction of the high 32 bits)."""
    total = int(np.prod(shape))
    span = np.uint64(hi - lo + 1)
    assert 0 < hi - lo + 1 <= (1 << 32)
    out = np.empty(total, dtype=dtype)
    with np.errstate(over="ignore"):
        for a, b in _rows(total):
            h = hash64(seed, tag, np.arange(a, b, dtype=np.uint64))
            v = ((h >> np.uint64(32)) * span) >> np.uint64(32)
            out[a:b] = (v.astype(np.int64) + lo).astype(dtype)
    return out.reshape(shape)


def uniform_f32(seed: int, tag: int, shape) -> np.ndarray:
    """FP32 uniform in [0, 1): multiples of 2^-24, so no denormals and no -0."""
    total = int(np.prod(shape))
    out = np.empty(total, dtype=np.float32)
    with np.errstate(over="ignore"):
        for a, b in _rows(total):
            h = hash64(seed, tag, np.arange(a, b, dtype=np.uint64))
            out[a:b] = ((h >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    return out.reshape(shape)


def uniform_unit_f64(seed: int, tag: int, idx: np.ndarray) -> np.ndarray:
    """Doubles uniform in [0, 1) with 53 random bits, for Bernoulli draws."""
    with np.errstate(over="ignore"):
        h = hash64(seed, tag, idx)
    return (h >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def random_graph(seed: int, tag: int, n: int, p: float, wlo: int, whi: int,
                 inf: int = INF_I32, dtype=np.int32) -> np.ndarray:
    """Weighted adjacency matrix of a random directed graph (Erdos-Renyi G(n, p)).

    W[i][i] = 0; an edge i->j (i != j) exists with probability p and has a
    weight uniform in [wlo, whi]; a missing edge is `inf`.  Edge draws use
    stream tag*2+1, weights stream tag*2.
    """
    total = n * n
    out = np.empty(total, dtype=dtype)
    span = np.uint64(whi - wlo + 1)
    with np.errstate(over="ignore"):
        for a, b in _rows(total):
            idx = np.arange(a, b, dtype=np.uint64)
            u = uniform_unit_f64(seed, 2 * tag + 1, idx)
            h = hash64(seed, 2 * tag, idx)
            w = (((h >> np.uint64(32)) * span) >> np.uint64(32)).astype(np.int64) + wlo
            i = idx // np.uint64(n)
            j = idx % np.uint64(n)
            v = np.where(u < p, w, inf)
            v = np.where(i == j, 0, v)
            out[a:b] = v.astype(dtype)
    return out.reshape(n, n)


def sample_indices(seed: int, tag: int, count: int, n: int) -> np.ndarray:
    """`count` distinct indices in [0, n), sorted (seeded; used for sampled rows)."""
    count = min(count, n)
    keys = hash64(seed, tag, np.arange(n, dtype=np.uint64))
    return np.sort(np.argsort(keys, kind="stable")[:count]).astype(np.int64)


def graph_sizes(seed: int, tag: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Instance sizes uniform in [lo, hi] for batched workloads."""
    return uniform_int(seed, tag, (count,), lo, hi, dtype=np.int64)


def loguniform_sizes(seed: int, tag: int, count: int, lo: int, hi: int) -> np.ndarray:
    """n = round(exp(U[ln lo, ln hi])) for the mixed serving workload."""
    u = uniform_unit_f64(seed, tag, np.arange(count, dtype=np.uint64))
    return np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
