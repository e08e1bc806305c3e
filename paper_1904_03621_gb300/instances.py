"""Seeded synthetic Ising instances.

This module only draws couplings J and fields h; it holds none of the
method's arithmetic, so both the CUDA path and the CPU oracle may use it.

The paper benchmarks "randomly generated" fully connected instances without
stating a generator (Sec. 3, Fig. 3 caption; Sec. 5.1).  The recipes below
stand in for them.  Every instance is drawn with ``numpy.random.default_rng``
(PCG64), in FP64 unless stated, returned as a dense symmetric n x n matrix
with zero diagonal (the library reads only its strict upper triangle).

Recipes (sizes and distributions of the five workloads):
  plain_n20      n=20, J_ij ~ N(0,1), h_i ~ N(0,1), seed 0, S=10
  int_n32        n=32, J_ij uniform in {-1,+1} (int32), h=0, seed 0, S=100
  float_n48      n=48, J_ij ~ N(0,1), h_i ~ N(0, 0.1^2) (std 0.1), seed 0, S=1000
  batched_4096   4096 instances, seed 0: 2048 dense (n ~ U{16..28},
                 J ~ N(0,1), h ~ N(0, 0.5^2)) then 2048 sparse Chimera
                 subgraphs (n ~ U{16..28}, J ~ U{-1,+1} on edges, h=0), S=10
  grad_256       256 instances n=28, J, h ~ N(0,1) cast to FP32, seed 0,
                 S=32, loss weights w ~ U(0,1) with seed 3
"""
from __future__ import annotations

import numpy as np


def _symmetric_from_upper(upper: np.ndarray) -> np.ndarray:
    J = np.triu(upper, 1)
    return J + J.T


def dense_gaussian(n: int, seed: int, h_std: float = 1.0, j_std: float = 1.0):
    """Fully connected instance: J_ij ~ N(0, j_std^2) (i<j), h_i ~ N(0, h_std^2)."""
    rng = np.random.default_rng(seed)
    J = _symmetric_from_upper(j_std * rng.standard_normal((n, n)))
    h = h_std * rng.standard_normal(n)
    return J.astype(np.float64), h.astype(np.float64)


def dense_pm1(n: int, seed: int):
    """Fully connected instance with J_ij uniform in {-1, +1} (int32) and h = 0."""
    rng = np.random.default_rng(seed)
    upper = (rng.integers(0, 2, size=(n, n)) * 2 - 1).astype(np.int32)
    J = _symmetric_from_upper(upper).astype(np.int32)
    h = np.zeros(n, dtype=np.int32)
    return J, h


def ferromagnet(n: int, dtype=np.int32):
    """J_ij = -1 for all pairs, h = 0 (ground states all-up / all-down under E)."""
    J = -np.ones((n, n), dtype=dtype)
    np.fill_diagonal(J, 0)
    return J, np.zeros(n, dtype=dtype)


def chimera_edges(rows: int, cols: int):
    """Edges (u, v), u < v, of a Chimera graph of rows x cols K_{4,4} cells.

    Vertex index v = ((r * cols + c) * 2 + shore) * 4 + t.  Inside a cell every
    shore-0 qubit couples to every shore-1 qubit; shore-0 qubit t couples to
    qubit t of the cell below, shore-1 qubit t to qubit t of the cell to the
    right.
    """
    def vid(r, c, k, t):
        return ((r * cols + c) * 2 + k) * 4 + t

    edges = []
    for r in range(rows):
        for c in range(cols):
            for t in range(4):
                for t2 in range(4):
                    edges.append((vid(r, c, 0, t), vid(r, c, 1, t2)))
                if r + 1 < rows:
                    edges.append((vid(r, c, 0, t), vid(r + 1, c, 0, t)))
                if c + 1 < cols:
                    edges.append((vid(r, c, 1, t), vid(r, c + 1, 1, t)))
    return sorted((min(u, v), max(u, v)) for u, v in edges)


def chimera_pm1(n: int, rng: np.random.Generator):
    """Induced subgraph on the first n vertices of a 2x2 or 2x3 Chimera grid
    (grid drawn uniformly), J = +-1 on its edges (int32), h = 0."""
    cols = 2 if rng.integers(0, 2) == 0 else 3
    edges = [(u, v) for (u, v) in chimera_edges(2, cols) if v < n]
    J = np.zeros((n, n), dtype=np.int32)
    vals = rng.integers(0, 2, size=len(edges)) * 2 - 1
    for (u, v), x in zip(edges, vals):
        J[u, v] = x
        J[v, u] = x
    return J, np.zeros(n, dtype=np.int32)


# ---- the five workloads ----------------------------------------------------

def plain_n20(seed: int = 0):
    return dense_gaussian(20, seed, h_std=1.0)


def int_n32(seed: int = 0):
    return dense_pm1(32, seed)


def float_n48(seed: int = 0):
    return dense_gaussian(48, seed, h_std=0.1)


def batched_4096(seed: int = 0, count: int = 4096, n_lo: int = 16, n_hi: int = 28):
    """List of (J, h, kind) with kind in {"dense", "sparse"}; first half dense."""
    rng = np.random.default_rng(seed)
    out = []
    half = count // 2
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        if i < half:
            J = _symmetric_from_upper(rng.standard_normal((n, n)))
            h = 0.5 * rng.standard_normal(n)
            out.append((J.astype(np.float64), h.astype(np.float64), "dense"))
        else:
            J, h = chimera_pm1(n, rng)
            out.append((J, h, "sparse"))
    return out


def grad_256(seed: int = 0, count: int = 256, n: int = 28, S: int = 32, w_seed: int = 3):
    """(list of (J, h) in FP32, weights w of shape (count, S))."""
    rng = np.random.default_rng(seed)
    inst = []
    for _ in range(count):
        J = _symmetric_from_upper(rng.standard_normal((n, n))).astype(np.float32)
        h = rng.standard_normal(n).astype(np.float32)
        inst.append((J, h))
    w = np.random.default_rng(w_seed).uniform(0.0, 1.0, size=(count, S))
    return inst, w


def pack(instances, dtype=np.float64):
    """Pack a list of (J, h, ...) into flat arrays + int64 element offsets.

    Integer couplings are carried exactly when dtype is float64.
    Returns (n, J_packed, J_off, h_packed, h_off).
    """
    n = np.array([np.asarray(t[0]).shape[0] for t in instances], dtype=np.int32)
    J_off = np.zeros(len(instances), dtype=np.int64)
    h_off = np.zeros(len(instances), dtype=np.int64)
    if len(instances) > 1:
        J_off[1:] = np.cumsum(n.astype(np.int64) ** 2)[:-1]
        h_off[1:] = np.cumsum(n.astype(np.int64))[:-1]
    J_packed = np.concatenate([np.asarray(t[0], dtype=dtype).ravel() for t in instances])
    h_packed = np.concatenate([np.asarray(t[1], dtype=dtype).ravel() for t in instances])
    return n, J_packed, J_off, h_packed, h_off
