"""The 10-spin unrolled walk (gray_kernel<10>) against the oracle, element by element.

By default the library walks 10 inner spins only in searches of at least 2^42
configurations, which the oracle cannot enumerate.  The inner_bits option forces
the block size, so the kernel that runs the full-size n = 48 search (its
per-walk task setup, its 1023-step increment table and its segment merges) is
compared here with the oracle on spaces the oracle enumerates: integers bit-exact,
floats within the tolerance of parity.py (1e-9 (sum|J| + sum|h|)).
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from parity import assert_float_parity, assert_int_equal
from paper_1904_03621_gb300 import instances

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
IB10 = {"inner_bits": 10}


@pytest.fixture(scope="module")
def bf():
    import torch
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import api
    assert torch.cuda.is_available()
    return api


@pytest.fixture(scope="module")
def o():
    return oracle.get()


def run(bf, J, h, S, **kw):
    import torch
    Jt = torch.as_tensor(np.ascontiguousarray(J)).cuda()
    ht = torch.as_tensor(np.ascontiguousarray(h)).cuda()
    en, st = bf.low_spectrum(Jt, ht, S, **kw)
    return en.cpu().numpy(), bf.states_u64(st)


def check(bf, o, J, h, S, **kw):
    en, st = run(bf, J, h, S, **kw)
    fb, fv = kw.get("fixed_bits", 0), kw.get("fixed_value", 0)
    n = np.asarray(J).shape[0]
    if np.issubdtype(np.asarray(J).dtype, np.integer):
        en_o, st_o = o.low_spectrum(J, h, S, fixed_bits=fb, fixed_value=fv)
        assert_int_equal(en, st, en_o, st_o)
    else:
        S1 = min(S + 1, 1 << (n - fb))
        Jd = np.asarray(J, dtype=np.float64)
        hd = np.asarray(h, dtype=np.float64)
        en_o, st_o = o.low_spectrum(Jd, hd, S1, fixed_bits=fb, fixed_value=fv)
        assert_float_parity(o, Jd, hd, en, st, en_o, st_o)
    return en, st


@pytest.mark.parametrize("n,S,seed", [(14, 7, 0), (20, 100, 1), (24, 1000, 2), (26, 2048, 3)])
def test_inner10_int_pm1(bf, o, n, S, seed):
    J, h = instances.dense_pm1(n, 500 + seed)
    check(bf, o, J, h, S, **IB10)


def test_inner10_int_wide_range(bf, o):
    rng = np.random.default_rng(22)
    n = 22
    U = rng.integers(-100000, 100000, (n, n))
    J = np.triu(U, 1)
    J = (J + J.T).astype(np.int32)
    h = rng.integers(-50000, 50000, n).astype(np.int32)
    check(bf, o, J, h, 64, **IB10)


def test_inner10_int_n32_full(bf):
    """n = 32, J uniform in {-1, +1}, h = 0, S = 100: bit-exact against the stored full enumeration."""
    import importlib.util
    path = os.path.join(GOLDEN, "int_n32_S100.txt.gz")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    gold = mg.read(path)
    J, h = instances.int_n32()
    en, st = run(bf, J, h, 100, **IB10)
    assert_int_equal(en, st, gold[0][0], gold[0][1])


@pytest.mark.parametrize("n,S,seed", [(14, 1, 0), (18, 2048, 1), (20, 1, 2), (22, 100, 3), (24, 2048, 4),
                                      (26, 100, 5)])
def test_inner10_float64(bf, o, n, S, seed):
    J, h = instances.dense_gaussian(n, 600 + seed)
    check(bf, o, J, h, S, **IB10)


def test_inner10_float32(bf, o):
    J, h = instances.dense_gaussian(21, 611)
    check(bf, o, J.astype(np.float32), h.astype(np.float32), 100, **IB10)


@pytest.mark.parametrize("n,fb,S", [(28, 4, 100), (30, 6, 2048), (30, 5, 1)])
def test_inner10_float_subspaces(bf, o, n, fb, S):
    """n = 28..30 in fixed-prefix subspaces of 2^24..2^25 configurations."""
    J, h = instances.dense_gaussian(n, 620 + n, h_std=0.1)
    for v in (0, (1 << fb) - 1, (1 << fb) // 3):
        check(bf, o, J, h, S, fixed_bits=fb, fixed_value=v, **IB10)


def test_inner10_ferromagnet(bf, o):
    for dt in (np.int32, np.float64):
        J, h = instances.ferromagnet(20, dtype=dt)
        check(bf, o, J, h, 100, **IB10)


def test_inner10_all_degenerate_ties(bf, o):
    """J = 0, h = 0: every configuration ties; the order is c = 0, 1, 2, ..."""
    n = 18
    for dt in (np.int32, np.float64):
        J = np.zeros((n, n), dtype=dt)
        h = np.zeros(n, dtype=dt)
        en, st = run(bf, J, h, 100, **IB10)
        assert list(st) == list(range(100)) and np.all(en == 0)


def test_inner10_spill_overflow_reports_status(bf):
    import torch
    from paper_1904_03621_gb300 import _lib
    n = 20
    J = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    h = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.BFError) as e:
        bf.low_spectrum(J, h, 10, spill_log2=4, **IB10)
    assert e.value.status == _lib.BF_EOVERFLOW
    en, st = bf.low_spectrum(J, h, 10, **IB10)
    assert bf.states_u64(st).tolist() == list(range(10))


@pytest.mark.parametrize("kw", [{}, {"task_log2": 12}, {"task_log2": 16, "grid_blocks": 3}, {"grid_blocks": 1},
                                {"task_log2": 22}, {"task_log2": 24, "grid_blocks": 2}])
def test_inner10_task_and_grid_options(bf, o, kw):
    """Tasks of 2^2..2^14 blocks (long tasks pass the dense and the every-16-blocks merges)."""
    J, h = instances.dense_gaussian(24, 640)
    check(bf, o, J, h, 300, **IB10, **kw)
    Ji, hi = instances.dense_pm1(24, 641)
    check(bf, o, Ji, hi, 300, **IB10, **kw)


def test_inner10_n64_subspace(bf, o):
    J, h = instances.dense_gaussian(64, 650)
    check(bf, o, J, h, 20, fixed_bits=42, fixed_value=(1 << 42) - 4321, **IB10)
    Ji, hi = instances.dense_pm1(64, 651)
    check(bf, o, Ji, hi, 20, fixed_bits=42, fixed_value=123456789, **IB10)


def test_inner10_float_n48_subspaces(bf, o):
    """The benchmark instance on all 64 stored fixed-prefix subspaces (top 24 bits fixed), S = 1000,
    walked with 10 inner spins as the full 2^48 search is."""
    import importlib.util
    path = os.path.join(GOLDEN, "float_n48_sub24_S1000.txt.gz")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    gold = mg.read(path)
    J, h = instances.float_n48()
    assert len(gold) == 64
    for v, (en_o, st_o) in sorted(gold.items()):
        en, st = run(bf, J, h, mg.N48_S, fixed_bits=mg.N48_FIXED_BITS, fixed_value=v, **IB10)
        assert_float_parity(o, J, h, en, st, en_o, st_o)


def test_inner10_equals_inner9_n36(bf):
    """Both block sizes give the same unique (E, c) list on a space too large for the oracle."""
    J, h = instances.dense_gaussian(36, 660, h_std=0.1)
    a = run(bf, J, h, 1000, inner_bits=9)
    b = run(bf, J, h, 1000, inner_bits=10)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])


def test_inner_bits_argument_checks(bf):
    import torch
    from paper_1904_03621_gb300 import _lib
    J = torch.zeros(13, 13, dtype=torch.float64, device="cuda")
    h = torch.zeros(13, dtype=torch.float64, device="cuda")
    for bad in ({"inner_bits": 10}, {"inner_bits": 8}, {"inner_bits": 11}):
        with pytest.raises(_lib.BFError) as e:
            bf.low_spectrum(J, h, 5, **bad)
        assert e.value.status == _lib.BF_EINVAL
