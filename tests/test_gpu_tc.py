"""The tensor-core screening variant (BF_VARIANT_TC) against the oracle and the Gray variant."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from parity import assert_float_parity, assert_int_equal
from paper_1904_03621_gb300 import instances

pytestmark = pytest.mark.gpu

TC = 2
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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
    en, st = bf.low_spectrum(torch.as_tensor(np.ascontiguousarray(J)).cuda(),
                             torch.as_tensor(np.ascontiguousarray(h)).cuda(), S, **kw)
    return en.cpu().numpy(), bf.states_u64(st)


def check(bf, o, J, h, S, **kw):
    en, st = run(bf, J, h, S, variant=TC, **kw)
    fb, fv = kw.get("fixed_bits", 0), kw.get("fixed_value", 0)
    n = np.asarray(J).shape[0]
    if np.issubdtype(np.asarray(J).dtype, np.integer):
        en_o, st_o = o.low_spectrum(J, h, S, fixed_bits=fb, fixed_value=fv)
        assert_int_equal(en, st, en_o, st_o)
    else:
        Jd, hd = np.asarray(J, dtype=np.float64), np.asarray(h, dtype=np.float64)
        en_o, st_o = o.low_spectrum(Jd, hd, min(S + 1, 1 << (n - fb)), fixed_bits=fb, fixed_value=fv)
        assert_float_parity(o, Jd, hd, en, st, en_o, st_o)
    return en, st


@pytest.mark.parametrize("n,S,seed", [(15, 1, 0), (15, 100, 1), (16, 10, 2), (18, 1000, 3), (20, 10, 4),
                                      (22, 100, 5), (24, 1000, 6)])
def test_tc_float(bf, o, n, S, seed):
    J, h = instances.dense_gaussian(n, seed)
    check(bf, o, J, h, S)


@pytest.mark.parametrize("n,S,seed", [(16, 17, 7), (20, 100, 8), (24, 2048, 9)])
def test_tc_int(bf, o, n, S, seed):
    J, h = instances.dense_pm1(n, seed)
    check(bf, o, J, h, S)


def test_tc_float32_and_subspace(bf, o):
    J, h = instances.dense_gaussian(30, 31)
    check(bf, o, J.astype(np.float32), h.astype(np.float32), 64, fixed_bits=8, fixed_value=77)
    Ji, hi = instances.dense_pm1(40, 12)
    check(bf, o, Ji, hi, 50, fixed_bits=18, fixed_value=12345)


def test_tc_task_sizes(bf, o):
    J, h = instances.dense_gaussian(26, 41)
    ref = None
    for kw in ({}, {"task_log2": 15}, {"task_log2": 18, "grid_blocks": 5}, {"grid_blocks": 1}):
        en, st = check(bf, o, J, h, 100, **kw)
        if ref is None:
            ref = st
        assert np.array_equal(st, ref)


def test_tc_ties_and_ferromagnet(bf, o):
    n = 18
    J = np.zeros((n, n))
    h = np.zeros(n)
    en, st = run(bf, J, h, 100, variant=TC)
    assert list(st) == list(range(100)) and np.all(en == 0)
    Jf, hf = instances.ferromagnet(20, dtype=np.int32)
    check(bf, o, Jf, hf, 100)


def test_tc_matches_gray_on_n48_subspaces(bf, o):
    """n = 48 float instance: the tensor-core and Gray variants agree on 8 of the stored
    fixed-prefix subspaces, and both match the stored oracle records."""
    import importlib.util
    path = os.path.join(GOLDEN, "float_n48_sub24_S1000.txt.gz")
    if not os.path.exists(path):
        pytest.skip("golden not generated")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    gold = mg.read(path)
    J, h = instances.float_n48()
    for v in sorted(gold)[:8]:
        en_t, st_t = run(bf, J, h, 1000, variant=TC, fixed_bits=24, fixed_value=v)
        en_g, st_g = run(bf, J, h, 1000, variant=1, fixed_bits=24, fixed_value=v)
        assert np.array_equal(st_t, st_g)
        assert_float_parity(o, J, h, en_t, st_t, gold[v][0], gold[v][1])


def test_tc_bounded_wait_reports_timeout(bf, o):
    """Failure detection without a GPU fault: with stall_test the MMA warps issue nothing, the
    epilogue's bounded waits (0.2 s) run out, the call reports BF_ETIMEOUT, and the same
    context then runs a correct search."""
    import time
    from paper_1904_03621_gb300 import _lib
    J, h = instances.dense_gaussian(20, 3)
    t0 = time.time()
    with pytest.raises(_lib.BFError) as err:
        run(bf, J, h, 10, variant=TC, stall_test=1)
    assert err.value.status == _lib.BF_ETIMEOUT
    assert time.time() - t0 < 30.0
    check(bf, o, J, h, 10)
