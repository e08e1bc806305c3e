"""Comparison of library results with the oracle.

Integer instances: energies and states must be identical (bit-exact).
Float instances: with tol = 1e-9 * (sum|J| + sum|h|) (upper triangle of J),
  - every energy agrees with the oracle's energy of the same rank within tol;
  - every returned state's oracle energy agrees with the returned energy within tol;
  - the returned states equal the oracle's wherever the gap between the
    S-th and (S+1)-th oracle energies exceeds tol (as sets), and positionally
    for ranks whose neighbours are separated by more than tol.
"""
from __future__ import annotations

import numpy as np


def tolerance(J, h) -> float:
    J = np.asarray(J, dtype=np.float64)
    return 1e-9 * (np.abs(np.triu(J, 1)).sum() + np.abs(np.asarray(h, dtype=np.float64)).sum())


def assert_int_equal(en_gpu, st_gpu, en_or, st_or):
    en_gpu = np.asarray(en_gpu)
    assert np.array_equal(en_gpu.astype(np.int64), np.asarray(en_or).astype(np.int64)), \
        f"energies differ at ranks {np.nonzero(en_gpu != en_or)[0][:10]}"
    assert np.array_equal(np.asarray(st_gpu, dtype=np.uint64), np.asarray(st_or, dtype=np.uint64)), \
        f"states differ at ranks {np.nonzero(np.asarray(st_gpu, np.uint64) != np.asarray(st_or, np.uint64))[0][:10]}"


def assert_float_parity(o, J, h, en_gpu, st_gpu, en_or_s1, st_or_s1, energy=None):
    """en_or_s1 / st_or_s1: oracle result with S + 1 records (or S when S = 2^n).

    energy(J, h, c): the oracle's value of one configuration (default: Eq. (1),
    o.energy; pass o.qubo_energy for the QUBO form, J = a, h = b)."""
    energy = energy or o.energy
    S = len(en_gpu)
    tol = tolerance(J, h)
    en_gpu = np.asarray(en_gpu, dtype=np.float64)
    st_gpu = np.asarray(st_gpu, dtype=np.uint64)
    en_or = np.asarray(en_or_s1[:S], dtype=np.float64)
    st_or = np.asarray(st_or_s1[:S], dtype=np.uint64)
    err = np.abs(en_gpu - en_or)
    assert err.max() <= tol, f"max energy error {err.max():.3e} > tol {tol:.3e} at rank {err.argmax()}"
    assert len(set(st_gpu.tolist())) == S, "duplicate states"
    for k in range(S):
        e = energy(J, h, int(st_gpu[k]))
        assert abs(e - en_gpu[k]) <= tol, f"rank {k}: state {st_gpu[k]} has E={e}, returned {en_gpu[k]}"
    assert np.all(np.diff(en_gpu) >= -tol), "energies not ascending"
    if len(en_or_s1) > S:
        gap = en_or_s1[S] - en_or_s1[S - 1]
        if gap > tol:
            assert set(st_gpu.tolist()) == set(st_or.tolist()), "state sets differ although the S-th gap exceeds tol"
    for k in range(S):
        lo = en_or[k] - (en_or[k - 1] if k > 0 else -np.inf)
        hi = (en_or_s1[k + 1] if k + 1 < len(en_or_s1) else np.inf) - en_or[k]
        if lo > tol and hi > tol:
            assert st_gpu[k] == st_or[k], f"rank {k}: state {st_gpu[k]} != oracle {st_or[k]}"
