"""The zero-field reduction the searches use, checked on the oracle alone (CPU).

With h = 0, Eq. (1) is even in s: E(c) = E(~c) with ~c = c ^ (2^n - 1).  The batched and the
single-instance searches then enumerate only the half space with spin n-1 at -1 and write the
S lowest (E, c) of the whole space from the half space's S lowest and their mirrors, level by
level: within one energy the half-space records in increasing c, then the mirrors in the
reverse order of their originals.  This test applies that rule to the oracle's half-space
result (its subspace mode, top bit fixed to 0) and compares with the oracle's enumeration of
all 2^n configurations, ties included.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1904_03621_gb300 import instances


def emit_with_mirrors(en, st, n, S):
    mirror = (1 << n) - 1
    out_e, out_c = [], []
    keep, i = len(en), 0
    while len(out_e) < S and i < keep:
        j = i + 1
        while j < keep and en[j] == en[i]:
            j += 1
        for t in range(i, j):
            if len(out_e) < S:
                out_e.append(en[t])
                out_c.append(int(st[t]))
        for t in range(j - 1, i - 1, -1):
            if len(out_e) < S:
                out_e.append(en[t])
                out_c.append(int(st[t]) ^ mirror)
        i = j
    return np.asarray(out_e), np.asarray(out_c, dtype=np.uint64)


def zero_field_instance(kind, n):
    if kind == "pm1":
        return instances.dense_pm1(n, 700 + n)
    if kind == "ferro":
        return instances.ferromagnet(n)
    J, h = instances.dense_gaussian(n, 710 + n)
    return J, np.zeros_like(h)


@pytest.mark.parametrize("kind,n,S", [("pm1", 10, 1), ("pm1", 12, 37), ("pm1", 14, 200), ("pm1", 16, 1000),
                                      ("ferro", 12, 90), ("gauss", 12, 64), ("gauss", 15, 300)])
def test_half_space_with_mirrors_is_the_full_spectrum(kind, n, S):
    o = oracle.get()
    J, h = zero_field_instance(kind, n)
    assert not np.any(h)
    en_full, st_full = o.low_spectrum(J, h, S)
    en_half, st_half = o.low_spectrum(J, h, S, fixed_bits=1, fixed_value=0)
    assert np.all(st_half < (1 << (n - 1)))
    en, st = emit_with_mirrors(en_half, st_half, n, S)
    assert np.array_equal(st, st_full)
    assert np.array_equal(en, en_full)


def test_mirror_energies_are_equal_with_zero_fields():
    """The premise: every configuration and its complement have the same energy when h = 0."""
    o = oracle.get()
    J, h = instances.dense_gaussian(11, 730)
    h = np.zeros_like(h)
    en, st = o.low_spectrum(J, h, 1 << 11)
    by_c = dict(zip((int(c) for c in st), en))
    mask = (1 << 11) - 1
    assert all(by_c[c] == by_c[c ^ mask] for c in by_c)
