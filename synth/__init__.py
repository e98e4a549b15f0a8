"""Seeded synthetic inputs for the semiring product and closure.

This module only draws inputs: edge sets and integer edge weights.  It holds
none of the method's arithmetic (no anti-distance encoding, no bit packing, no
semiring operation); both the CUDA path and the CPU oracle take its arrays and
encode them themselves.

Every draw comes from one counter-based hash, so any entry of any matrix can be
regenerated on its own, in any order, on any machine:

    sm64(x)             = splitmix64 finaliser (Steele, Lea & Flood, 2014,
                          "Fast splittable pseudorandom number generators"):
                          z = x + 0x9E3779B97F4A7C15
                          z = (z ^ z>>30) * 0xBF58476D1CE4E5B9
                          z = (z ^ z>>27) * 0x94D049BB133111EB
                          return z ^ z>>31            (all mod 2**64)
    h(seed, s, i, j)    = sm64(sm64(sm64(seed * K1 + s) + i) + j)

An edge (i, j) is present iff h(seed, s_edge, i, j) < floor(p * 2**64); its
weight is lo + h(seed, s_edge + 1, i, j) mod (hi - lo + 1).

Weight matrices use 0 for "no edge" (generated weights are >= 1).  Boolean
matrices are dense uint8 0/1 arrays (row-major, entry (i, j) = edge i -> j).
"""

from __future__ import annotations

from fractions import Fraction
import math

import numpy as np

__all__ = [
    "sm64", "hash_grid", "threshold", "bernoulli", "weighted_graph",
    "bool_dag_union", "log_uniform_sizes", "graph_seed",
    "cfg1_bool_product", "cfg2_antidist", "cfg3_bool_closure", "cfg4_batched",
]

_M64 = (1 << 64) - 1
K1 = 0xD1B54A32D192ED03
_G = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def _sm64_int(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def sm64(x):
    """splitmix64 finaliser on a python int or a uint64 numpy array."""
    if isinstance(x, (int, np.integer)):
        return _sm64_int(int(x) & _M64)
    z = np.asarray(x, dtype=np.uint64) + _G
    z = (z ^ (z >> np.uint64(30))) * _C1
    z = (z ^ (z >> np.uint64(27))) * _C2
    return z ^ (z >> np.uint64(31))


def h_int(seed: int, s: int, i: int, j: int) -> int:
    """Scalar form of the hash, for spot checks of single entries."""
    return _sm64_int((_sm64_int((_sm64_int((seed * K1 + s) & _M64) + i) & _M64) + j) & _M64)


def hash_grid(seed: int, s: int, rows, cols) -> np.ndarray:
    """h(seed, s, i, j) for i in rows, j in cols, as a (len(rows), len(cols)) uint64 array."""
    rows = np.asarray(rows, dtype=np.uint64)
    cols = np.asarray(cols, dtype=np.uint64)
    base = np.uint64(_sm64_int((seed * K1 + s) & _M64))
    with np.errstate(over="ignore"):
        hr = sm64(base + rows)                      # one value per row
        return sm64(hr[:, None] + cols[None, :])


def threshold(p: float) -> int:
    """floor(p * 2**64) computed exactly from the binary value of p."""
    if p <= 0:
        return 0
    if p >= 1:
        return 1 << 64
    return int(Fraction(p) * (1 << 64))


def _chunks(n: int, step: int):
    for r0 in range(0, n, step):
        yield r0, min(n, r0 + step)


def bernoulli(R: int, C: int, p: float, seed: int, s: int, diag: bool = True,
              chunk: int = 1024) -> np.ndarray:
    """Dense uint8 0/1 matrix, entry (i, j) = 1 w.p. p; diagonal zeroed unless diag."""
    thr = threshold(p)
    out = np.zeros((R, C), dtype=np.uint8)
    cols = np.arange(C)
    for r0, r1 in _chunks(R, chunk):
        hg = hash_grid(seed, s, np.arange(r0, r1), cols)
        if thr >= (1 << 64):
            blk = np.ones_like(hg, dtype=np.uint8)
        else:
            blk = (hg < np.uint64(thr)).astype(np.uint8)
        out[r0:r1] = blk
    if not diag:
        n = min(R, C)
        out[np.arange(n), np.arange(n)] = 0
    return out


def weighted_graph(R: int, C: int, p: float, wlo: int, whi: int, seed: int, s_edge: int,
                   dtype=np.uint8, diag: bool = False, chunk: int = 1024) -> np.ndarray:
    """Weight matrix: W[i, j] in [wlo, whi] for an edge, 0 for no edge."""
    assert 1 <= wlo <= whi
    thr = threshold(p)
    span = np.uint64(whi - wlo + 1)
    out = np.zeros((R, C), dtype=dtype)
    cols = np.arange(C)
    for r0, r1 in _chunks(R, chunk):
        rows = np.arange(r0, r1)
        e = hash_grid(seed, s_edge, rows, cols) < np.uint64(min(thr, _M64))
        if thr >= (1 << 64):
            e[:] = True
        w = (hash_grid(seed, s_edge + 1, rows, cols) % span).astype(np.int64) + wlo
        out[r0:r1] = np.where(e, w, 0).astype(dtype)
    if not diag:
        n = min(R, C)
        out[np.arange(n), np.arange(n)] = 0
    return out


def bool_dag_union(D: int, seed: int, p_dag: float | None = None, p_rand: float | None = None,
                   chunk: int = 1024) -> np.ndarray:
    """Union of a random DAG (i -> j, i < j, w.p. 2/D) and a random digraph with
    mean out-degree 1.5 (i -> j, i != j, w.p. 1.5/D).  Dense uint8 0/1."""
    p_dag = 2.0 / D if p_dag is None else p_dag
    p_rand = 1.5 / D if p_rand is None else p_rand
    t_dag, t_rand = np.uint64(threshold(p_dag)), np.uint64(threshold(p_rand))
    out = np.zeros((D, D), dtype=np.uint8)
    cols = np.arange(D)
    for r0, r1 in _chunks(D, chunk):
        rows = np.arange(r0, r1)
        dag = (hash_grid(seed, 0, rows, cols) < t_dag) & (rows[:, None] < cols[None, :])
        rnd = (hash_grid(seed, 5, rows, cols) < t_rand) & (rows[:, None] != cols[None, :])
        out[r0:r1] = (dag | rnd).astype(np.uint8)
    return out


def log_uniform_sizes(n: int, lo: int, hi: int, seed: int, s: int = 2) -> list[int]:
    """D_g = clamp(round(lo * (hi/lo)**u_g), lo, hi), u_g = (h(seed, s, g, 0) >> 11) * 2**-53."""
    out = []
    for g in range(n):
        u = (h_int(seed, s, g, 0) >> 11) * 2.0 ** -53
        out.append(int(min(hi, max(lo, round(lo * (hi / lo) ** u)))))
    return out


def graph_seed(seed: int, g: int) -> int:
    """Seed of graph g within a batch (or request g of a stream)."""
    return h_int(seed, 7, g, 0) & ((1 << 62) - 1)


# ---------------------------------------------------------------------------
# Workloads (shapes, densities and weight ranges of the five configurations)
# ---------------------------------------------------------------------------

def cfg1_bool_product(R: int = 512, K: int = 512, N: int = 512, p: float = 0.02, seed: int = 0):
    """Boolean product operands: A (R x K) from stream 0, B (K x N) from stream 1."""
    A = bernoulli(R, K, p, seed, 0, diag=True)
    B = bernoulli(K, N, p, seed, 1, diag=True)
    return A, B


def cfg2_antidist(D: int = 4096, p: float = 0.05, wlo: int = 1, whi: int = 31, seed: int = 1,
                  s_edge: int = 0, dtype=np.uint8) -> np.ndarray:
    """Weighted digraph, no self-loops; product operands use s_edge = 0 (A) and 3 (B)."""
    return weighted_graph(D, D, p, wlo, whi, seed, s_edge, dtype=dtype, diag=False)


def cfg3_bool_closure(D: int = 16384, seed: int = 2) -> np.ndarray:
    return bool_dag_union(D, seed)


def cfg4_batched(n: int = 2000, lo: int = 32, hi: int = 1024, seed: int = 3,
                 wlo: int = 1, whi: int = 4000):
    """(sizes, list of uint16 weight matrices), density 8/D per graph."""
    sizes = log_uniform_sizes(n, lo, hi, seed)
    mats = [weighted_graph(D, D, min(1.0, 8.0 / D), wlo, whi, graph_seed(seed, g), 0,
                           dtype=np.uint16, diag=False) for g, D in enumerate(sizes)]
    return sizes, mats


def expected_log_uniform_cube(lo: int, hi: int) -> float:
    """E[D^3] for D log-uniform on [lo, hi] (continuous), used for sanity checks."""
    return (hi ** 3 - lo ** 3) / (3 * math.log(hi / lo))
