"""Pins of the CPU oracle against facts that do not come from the oracle.

Each ``pin_*`` function takes an ``oracle.Oracle`` handle and raises
AssertionError when the oracle disagrees with the paper, a closed form, an
invariant of Eq. (1) or an independent library computation.  The same
functions run against copies of the oracle with planted mistakes
(test_oracle_mutants.py) to show that each class of mistake is caught.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _spins(n):
    """All 2^n spin vectors, row c = configuration integer c, LSB = spin 0."""
    c = np.arange(1 << n, dtype=np.int64)
    return (((c[:, None] >> np.arange(n)) & 1) * 2 - 1).astype(np.float64)


def _garbage_lower(J, rng, scale=5.0):
    """Fill the diagonal and lower triangle with values that must be ignored."""
    J = np.array(J, dtype=np.float64, copy=True)
    n = J.shape[0]
    low = np.tril_indices(n)
    J[low] = scale * rng.standard_normal(len(low[0]))
    return J


# -- the paper's own examples -----------------------------------------------

def pin_paper_example(o):
    """Sec. 4.1 listing input, energies derived by hand (tests/golden/paper_example.txt)."""
    rows = _read_golden("paper_example.txt")
    n = int(rows[0][1])
    h = np.array([float(x) for x in rows[1][1:]])
    J01 = float(rows[2][1])
    # garbage on the diagonal and below it: the library reads only i < j
    J = np.array([[7.5, J01], [-3.25, 11.0]])
    want = [(float(r[1]), int(r[2])) for r in rows[3:]]
    for e_want, c in want:
        e = o.energy(J, h, c)
        assert abs(e - e_want) < 1e-12, f"E({c}) = {e}, expected {e_want}"
    en, st = o.low_spectrum(J, h, 4)
    assert [int(x) for x in st] == [c for _, c in want], f"order {st}"
    assert np.allclose(en, [e for e, _ in want], atol=1e-12, rtol=0)
    # the same instance with integer-scaled values (x5): exact in int64
    Ji = np.array([[9, -1], [4, -6]], dtype=np.int32)
    hi = np.array([-5, 0], dtype=np.int32)
    for e_want, c in want:
        assert o.energy(Ji, hi, c) == round(5 * e_want)


def pin_coding_example(o):
    """Sec. 3, Eq. (5): #13 = (00001101)_2 and the closed form E = 2c - (2^n - 1)
    for J = 0, h_i = 2^i (tests/golden/coding_example.txt)."""
    rows = _read_golden("coding_example.txt")
    n = int(rows[0][1])
    c13 = int(rows[1][1])
    spins = [int(x) for x in rows[2][1:]]
    e13 = int(rows[3][1])
    h = np.array([2.0 ** i for i in range(n)])
    J = np.zeros((n, n))
    assert o.energy(J, h, c13) == float(e13)
    # each spin of #13 individually: a field on one spin reads its value
    for i, s in enumerate(spins):
        hi = np.zeros(n)
        hi[i] = 1.0
        assert o.energy(J, hi, c13) == float(s), f"spin {i}"
    for c in range(1 << n):
        assert o.energy(J, h, c) == float(2 * c - ((1 << n) - 1))


# -- closed forms ----------------------------------------------------------

def ferromagnet_energy(n, c):
    """J_ij = -1 (all pairs), h = 0: E = -((sum s)^2 - n) / 2, sum s = 2 popcount(c) - n."""
    m = 2 * bin(c).count("1") - n
    return -(m * m - n) // 2


def pin_ferromagnet(o):
    for n in (3, 7, 10):
        J = -np.ones((n, n), dtype=np.int32)
        h = np.zeros(n, dtype=np.int32)
        all_e = o.all_energies(J, h)
        want = np.array([ferromagnet_energy(n, c) for c in range(1 << n)])
        assert np.array_equal(all_e, want), f"ferromagnet n={n}"
        # lowest levels: E_0 = -n(n-1)/2 at c = 0 and 2^n - 1, then single flips
        S = 2 + 2 * n
        en, st = o.low_spectrum(J, h, S)
        assert en[0] == -n * (n - 1) // 2 and list(st[:2]) == [0, (1 << n) - 1]
        e1 = -((n - 2) ** 2 - n) // 2
        assert all(x == e1 for x in en[2:])
        singles = sorted([1 << i for i in range(n)] + [((1 << n) - 1) ^ (1 << i) for i in range(n)])
        assert [int(x) for x in st[2:]] == singles
        # float copy of the same instance
        ef, sf = o.low_spectrum(J.astype(np.float64), h.astype(np.float64), S)
        assert np.array_equal(ef, en.astype(np.float64)) and np.array_equal(sf, st)


def pin_fields_only(o):
    """J = 0: the spectrum is {sum_i +-|h_i|}; ground state s_i = -sign(h_i)."""
    rng = np.random.default_rng(11)
    n = 9
    h = rng.standard_normal(n)
    J = np.zeros((n, n))
    all_e = o.all_energies(J, h)
    want = np.array([sum(h[i] * (1 if (c >> i) & 1 else -1) for i in range(n)) for c in range(1 << n)])
    assert np.allclose(all_e, want, atol=1e-12, rtol=0)
    en, st = o.low_spectrum(J, h, 3)
    gs = sum(1 << i for i in range(n) if h[i] < 0)
    assert int(st[0]) == gs and abs(en[0] + np.abs(h).sum()) < 1e-12


# -- invariants of Eq. (1) ---------------------------------------------------

def pin_z2(o):
    """h = 0: E(c) = E(c xor (2^n - 1)); every level has even multiplicity."""
    rng = np.random.default_rng(5)
    n = 11
    J = rng.standard_normal((n, n))
    h = np.zeros(n)
    e = o.all_energies(J, h)
    mask = (1 << n) - 1
    assert np.array_equal(e, e[np.arange(1 << n) ^ mask])
    Ji = (rng.integers(0, 2, (n, n)) * 2 - 1).astype(np.int32)
    ei = o.all_energies(Ji, np.zeros(n, dtype=np.int32))
    _, counts = np.unique(ei, return_counts=True)
    assert np.all(counts % 2 == 0)


def pin_gauge(o):
    """s_i -> eps_i s_i, J_ij -> eps_i eps_j J_ij, h_i -> eps_i h_i leaves E invariant;
    states map by c' = c xor mask(eps = -1)."""
    rng = np.random.default_rng(6)
    n = 10
    J = rng.standard_normal((n, n))
    h = rng.standard_normal(n)
    eps = rng.integers(0, 2, n) * 2 - 1
    Jg = J * np.outer(eps, eps)
    hg = h * eps
    mask = sum(1 << i for i in range(n) if eps[i] < 0)
    e = o.all_energies(J, h)
    eg = o.all_energies(Jg, hg)
    assert np.array_equal(e, eg[np.arange(1 << n) ^ mask])
    S = 20
    en, st = o.low_spectrum(J, h, S)
    eng, stg = o.low_spectrum(Jg, hg, S)
    assert np.array_equal(en, eng)
    assert sorted(int(x) ^ mask for x in stg) == sorted(int(x) for x in st)


def pin_qubo(o):
    """Sec. 2, Eqs. (2)-(3): with the paper's sign (J_p = -J, h_p = -h),
    H(s) - F(q) = sum_i h_p,i - sum_{i<j} J_p,ij, where
    F(q) = -sum_{i<j} a_ij q_i q_j - sum_i b_i q_i, a = 4 J_p, b_i = 2 h_p,i - 2 sum_{j != i} J_p,ij."""
    rng = np.random.default_rng(7)
    n = 10
    J = rng.standard_normal((n, n))
    h = rng.standard_normal(n)
    U = np.triu(J, 1)
    Jp = -(U + U.T)
    hp = -h
    a = 4.0 * np.triu(Jp, 1)
    b = 2.0 * hp - 2.0 * Jp.sum(axis=1)
    offset = hp.sum() - np.triu(Jp, 1).sum()
    e = o.all_energies(J, h)
    for c in range(1 << n):
        q = np.array([(c >> i) & 1 for i in range(n)], dtype=np.float64)
        F = -(q @ a @ q) - b @ q
        assert abs(e[c] - (F + offset)) < 1e-10, f"c={c}"


def pin_sum_zero(o):
    """sum over all configurations of E(c) = 0 (every term is odd in some spin)."""
    rng = np.random.default_rng(8)
    for n in (5, 13):
        J = rng.standard_normal((n, n))
        h = rng.standard_normal(n)
        assert abs(o.all_energies(J, h).sum()) < 1e-8 * (1 << n)


def pin_matrix_form(o):
    """Explicit listing against numpy: E = s^T triu(J, 1) s + h . s, with garbage
    on and below the diagonal that must be ignored."""
    rng = np.random.default_rng(9)
    for n in (1, 2, 6, 8):
        J = _garbage_lower(rng.standard_normal((n, n)), rng)
        h = rng.standard_normal(n)
        Sm = _spins(n)
        want = np.einsum("ci,ij,cj->c", Sm, np.triu(J, 1), Sm) + Sm @ h
        assert np.allclose(o.all_energies(J, h), want, atol=1e-10, rtol=0), f"n={n}"
        Ji = (rng.integers(-9, 10, (n, n))).astype(np.int32)
        hi = rng.integers(-9, 10, n).astype(np.int32)
        wanti = np.einsum("ci,ij,cj->c", Sm, np.triu(Ji, 1).astype(np.float64), Sm) + Sm @ hi
        assert np.array_equal(o.all_energies(Ji, hi), wanti.astype(np.int64))


# -- selection (Algorithm 1 contract with (E, c) ties) -------------------------

def pin_full_sort(o):
    """S = 2^n returns every configuration sorted by (E, c): compare with numpy lexsort."""
    rng = np.random.default_rng(10)
    n = 10
    J = rng.standard_normal((n, n))
    h = rng.standard_normal(n)
    e = o.all_energies(J, h)
    order = np.lexsort((np.arange(1 << n), e))
    en, st = o.low_spectrum(J, h, 1 << n)
    assert np.array_equal(st, order.astype(np.uint64)) and np.array_equal(en, e[order])
    Ji = (rng.integers(0, 2, (n, n)) * 2 - 1).astype(np.int32)  # massive degeneracy
    hi = np.zeros(n, dtype=np.int32)
    ei = o.all_energies(Ji, hi)
    orderi = np.lexsort((np.arange(1 << n), ei))
    for S in (1, 37, 1 << n):
        en, st = o.low_spectrum(Ji, hi, S)
        assert np.array_equal(st, orderi[:S].astype(np.uint64)), f"S={S}"
        assert np.array_equal(en, ei[orderi[:S]])


def pin_ties(o):
    """All energies equal (J = 0, h = 0): the S lowest are c = 0 .. S-1."""
    n = 12
    for J, h in ((np.zeros((n, n)), np.zeros(n)), (np.zeros((n, n), np.int32), np.zeros(n, np.int32))):
        en, st = o.low_spectrum(J, h, 50)
        assert list(st) == list(range(50)) and np.all(en == 0)


def pin_streaming_equals_sort(o):
    """Per-thread bounded heaps give the same records as materialise-and-sort."""
    rng = np.random.default_rng(12)
    n = 18
    J = rng.standard_normal((n, n))
    h = rng.standard_normal(n)
    Ji = (rng.integers(0, 2, (n, n)) * 2 - 1).astype(np.int32)
    hi = np.zeros(n, dtype=np.int32)
    for S in (1, 7, 100):
        for JJ, hh in ((J, h), (Ji, hi)):
            a = o.low_spectrum(JJ, hh, S, mode=1)
            b = o.low_spectrum(JJ, hh, S, mode=2)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), f"S={S}"


def pin_subspace(o):
    """Sec. 3, Eq. (6): a fixed offset on the top bits enumerates exactly that chunk."""
    rng = np.random.default_rng(13)
    n, fb = 12, 4
    J = rng.standard_normal((n, n))
    h = rng.standard_normal(n)
    e = o.all_energies(J, h)
    for v in (0, 5, 15):
        cs = np.arange(v << (n - fb), (v + 1) << (n - fb))
        order = cs[np.lexsort((cs, e[cs]))]
        en, st = o.low_spectrum(J, h, 25, fixed_bits=fb, fixed_value=v)
        assert np.array_equal(st, order[:25].astype(np.uint64))


# -- gradient ----------------------------------------------------------------

def pin_grad(o):
    """dL/dJ_ij and dL/dh_i of L = sum_k g_k E(s_k) against central finite
    differences of the (separately pinned) energy."""
    rng = np.random.default_rng(14)
    n_list = [5, 7]
    S = 6
    states = [rng.integers(0, 1 << n, S, dtype=np.uint64) for n in n_list]
    g = rng.uniform(0, 1, (len(n_list), S))
    dJ, dh, J_off, h_off = o.grad(n_list, np.stack(states), g)
    step = 1e-3
    for b, n in enumerate(n_list):
        J = rng.standard_normal((n, n))
        h = rng.standard_normal(n)

        def L(JJ, hh):
            return sum(g[b, k] * o.energy(JJ, hh, int(states[b][k])) for k in range(S))

        Gj = dJ[J_off[b]:J_off[b] + n * n].reshape(n, n)
        for i, j in itertools.product(range(n), range(n)):
            if i < j:
                Jp, Jm = J.copy(), J.copy()
                Jp[i, j] += step
                Jm[i, j] -= step
                fd = (L(Jp, h) - L(Jm, h)) / (2 * step)
                assert abs(fd - Gj[i, j]) < 1e-8, f"dJ[{i},{j}]"
            else:
                assert Gj[i, j] == 0.0
        for i in range(n):
            hp_, hm_ = h.copy(), h.copy()
            hp_[i] += step
            hm_[i] -= step
            fd = (L(J, hp_) - L(J, hm_)) / (2 * step)
            assert abs(fd - dh[h_off[b] + i]) < 1e-8, f"dh[{i}]"


def _qubo_instance(rng, n, integer):
    """Random QUBO coefficients with junk on the diagonal and lower triangle of a
    (which Eq. (2)'s pair sum over i < j must ignore)."""
    if integer:
        a = rng.integers(-9, 10, (n, n)).astype(np.int32)
        b = rng.integers(-9, 10, n).astype(np.int32)
    else:
        a = rng.standard_normal((n, n))
        b = rng.standard_normal(n)
    return a, b


def pin_qubo_closed_forms(o):
    """Sec. 2, Eq. (2) (library sign) at configurations where the sum collapses:
    F(0) = 0, F(e_i) = b_i, F(e_i + e_j) = a_ij + b_i + b_j (i < j)."""
    rng = np.random.default_rng(21)
    for integer in (True, False):
        n = 9
        a, b = _qubo_instance(rng, n, integer)
        assert o.qubo_energy(a, b, 0) == 0
        for i in range(n):
            assert o.qubo_energy(a, b, 1 << i) == b[i]
            for j in range(i + 1, n):
                want = a[i, j] + b[i] + b[j]
                got = o.qubo_energy(a, b, (1 << i) | (1 << j))
                assert (got == want) if integer else abs(got - want) < 1e-12, (i, j)


def pin_qubo_ising_map(o):
    """Sec. 2, Eq. (3): with J_ij = a_ij / 4 (i < j) and h_i = b_i / 2 + sum_{j != i} a_ij / 4
    (library sign), E(s) - F(q) = sum_{i<j} J_ij - sum_i h_i for every configuration; the
    low spectra agree configuration by configuration (the offset is a constant)."""
    rng = np.random.default_rng(22)
    n = 10
    a, b = _qubo_instance(rng, n, integer=False)
    U = np.triu(a, 1)
    J = U / 4.0
    h = b / 2.0 + (U + U.T).sum(axis=1) / 4.0
    offset = np.triu(J, 1).sum() - h.sum()
    e = o.all_energies(J, h)
    for c in range(1 << n):
        assert abs(e[c] - o.qubo_energy(a, b, c) - offset) < 1e-10, c
    f_q, c_q = o.qubo_low_spectrum(a, b, 40)
    e_i, c_i = o.low_spectrum(J, h, 40)
    assert np.array_equal(c_q, c_i)
    assert np.abs((e_i - offset) - f_q).max() < 1e-10


def pin_qubo_separable(o):
    """a = 0: F(q) = sum_i b_i q_i, minimised by q_i = [b_i < 0] with value sum of the
    negative b_i; the next state flips the b_i of smallest magnitude."""
    rng = np.random.default_rng(23)
    n = 12
    b = rng.standard_normal(n)
    a = np.zeros((n, n))
    f, c = o.qubo_low_spectrum(a, b, 2)
    mask = sum(1 << i for i in range(n) if b[i] < 0)
    assert c[0] == mask and abs(f[0] - b[b < 0].sum()) < 1e-12
    k = int(np.argmin(np.abs(b)))
    assert c[1] == mask ^ (1 << k) and abs(f[1] - (f[0] + abs(b[k]))) < 1e-12


def pin_potts_q2_is_ising(o):
    """q = 2 Potts model (Sec. 2's extension to other classical models) against the Ising
    oracle: [s_i == s_j] = (1 + s_i s_j) / 2 and h_i(v) splits into its mean and its half
    difference, so E_P(c) = E_I(c; J/2, (h_i(1) - h_i(0)) / 2) + sum_{i<j} J_ij / 2 +
    sum_i (h_i(0) + h_i(1)) / 2 for every configuration (same bit encoding)."""
    rng = np.random.default_rng(31)
    n = 11
    J = rng.standard_normal((n, n))
    hp = rng.standard_normal((n, 2))
    U = np.triu(J, 1)
    e_i = o.all_energies(U / 2.0, (hp[:, 1] - hp[:, 0]) / 2.0)
    const = U.sum() / 2.0 + hp.sum() / 2.0
    for c in range(1 << n):
        assert abs(o.potts_energy(J, hp, c) - (e_i[c] + const)) < 1e-10, c
    e_p, c_p = o.potts_low_spectrum(J, hp, 30)
    e_s, c_s = o.low_spectrum(U / 2.0, (hp[:, 1] - hp[:, 0]) / 2.0, 30)
    assert np.array_equal(c_p, c_s) and np.abs(e_p - (e_s + const)).max() < 1e-10


def pin_potts_ferromagnet(o):
    """J_ij = -1, h = 0: the q uniform configurations c = v (q^n - 1) / (q - 1) are the ground
    states with E = -n(n-1)/2; the next level, one spin different, has E = -(n-1)(n-2)/2 and
    multiplicity n q (q - 1)."""
    for n, q in ((6, 3), (5, 4)):
        J = -np.ones((n, n), dtype=np.int32)
        h = np.zeros((n, q), dtype=np.int32)
        k = q + n * q * (q - 1)
        e, c = o.potts_low_spectrum(J, h, k + 1)
        rep = (q ** n - 1) // (q - 1)
        assert list(c[:q]) == [v * rep for v in range(q)]
        assert all(e[:q] == -n * (n - 1) // 2)
        assert all(e[q:k] == -(n - 1) * (n - 2) // 2)
        assert e[k] > e[k - 1]


def pin_potts_fields_only(o):
    """J = 0: E = sum_i h_i(sigma_i) is separable; the ground state takes argmin_v h_i(v)
    per spin and the next state changes the spin with the smallest second-best gap."""
    rng = np.random.default_rng(32)
    n, q = 7, 3
    h = rng.standard_normal((n, q))
    J = np.zeros((n, n))
    e, c = o.potts_low_spectrum(J, h, 2)
    best = h.argmin(axis=1)
    assert c[0] == sum(int(best[i]) * q ** i for i in range(n))
    assert abs(e[0] - h.min(axis=1).sum()) < 1e-12
    srt = np.sort(h, axis=1)
    gaps = srt[:, 1] - srt[:, 0]
    assert abs(e[1] - (e[0] + gaps.min())) < 1e-12


def pin_potts_relabel_and_sum(o):
    """h = 0: a global relabelling of the q states leaves E unchanged.  With fields: the sum of
    E over all q^n configurations is q^(n-1) (sum_{i<j} J_ij + sum_{i,v} h_i(v))."""
    rng = np.random.default_rng(33)
    n, q = 6, 3
    J = rng.integers(-5, 6, (n, n)).astype(np.int32)
    h0 = np.zeros((n, q), dtype=np.int32)
    perm = [2, 0, 1]
    for c in rng.integers(0, q ** n, 40):
        d = [(int(c) // q ** i) % q for i in range(n)]
        c2 = sum(perm[d[i]] * q ** i for i in range(n))
        assert o.potts_energy(J, h0, int(c)) == o.potts_energy(J, h0, c2)
    h = rng.integers(-5, 6, (n, q)).astype(np.int32)
    total = sum(o.potts_energy(J, h, c) for c in range(q ** n))
    assert total == q ** (n - 1) * (int(np.triu(J, 1).sum()) + int(h.sum()))


ALL_PINS = [
    pin_paper_example, pin_coding_example, pin_ferromagnet, pin_fields_only, pin_z2, pin_gauge,
    pin_qubo, pin_sum_zero, pin_matrix_form, pin_full_sort, pin_ties, pin_streaming_equals_sort,
    pin_subspace, pin_grad, pin_qubo_closed_forms, pin_qubo_ising_map, pin_qubo_separable,
    pin_potts_q2_is_ising, pin_potts_ferromagnet, pin_potts_fields_only, pin_potts_relabel_and_sum,
]
