"""bf_autotune: the single-instance search's kernel and launch shape chosen by timing candidates
on this GPU.  The choice must be a valid option set, it must be cached and used by later default
calls, and results must not depend on it: the tuned default gives exactly the result of explicit
options and of the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from parity import assert_float_parity, assert_int_equal
from paper_1904_03621_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    import torch
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import api
    assert torch.cuda.is_available()
    return api


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_choice(t, n, free_bits):
    assert t["variant"] in (1, 2)
    if t["variant"] == 1:
        assert t["inner_bits"] in (9, 10) and t["grid_blocks"] > 0 and t["task_log2"] >= t["inner_bits"]
    else:
        assert free_bits >= 15 and t["task_log2"] >= 15
    assert t["configs_per_s"] > 0


@pytest.mark.parametrize("kind,n,S", [("float", 24, 100), ("int", 26, 500), ("float", 30, 1000)])
def test_autotune_default_equals_explicit_and_oracle(bf, kind, n, S):
    o = oracle.get()
    J, h = (instances.dense_gaussian if kind == "float" else instances.dense_pm1)(n, 1100 + n)
    Jd, hd = dev(J), dev(h)
    t = bf.autotune(Jd, hd, S)
    check_choice(t, n, n)
    en_t, st_t = bf.low_spectrum(Jd, hd, S)                 # default options: the cached choice
    en_x, st_x = bf.low_spectrum(Jd, hd, S, variant=1, inner_bits=9, task_log2=12, grid_blocks=100)
    assert np.array_equal(bf.states_u64(st_t), bf.states_u64(st_x))
    assert np.array_equal(en_t.cpu().numpy(), en_x.cpu().numpy())
    if kind == "int":
        assert_int_equal(en_t.cpu().numpy(), bf.states_u64(st_t), *o.low_spectrum(J, h, S))
    elif n <= 26:
        assert_float_parity(o, J, h, en_t.cpu().numpy(), bf.states_u64(st_t), *o.low_spectrum(J, h, S + 1))


def test_autotune_large_space_times_a_part_of_the_queue(bf):
    """2^40 configurations (n = 42, top 2 bits fixed): the tuner times the last 2^39 of the task
    queue per candidate; the tuned default search equals the explicit-option search."""
    J, h = instances.dense_gaussian(42, 1200, h_std=0.1)
    Jd, hd = dev(J), dev(h)
    t = bf.autotune(Jd, hd, 200, fixed_bits=2, fixed_value=1)
    check_choice(t, 42, 40)
    en_t, st_t = bf.low_spectrum(Jd, hd, 200, fixed_bits=2, fixed_value=1)
    en_x, st_x = bf.low_spectrum(Jd, hd, 200, fixed_bits=2, fixed_value=1, variant=1, inner_bits=10)
    assert np.array_equal(bf.states_u64(st_t), bf.states_u64(st_x))
    assert np.array_equal(en_t.cpu().numpy(), en_x.cpu().numpy())


def test_autotune_tiny_space(bf):
    o = oracle.get()
    J, h = instances.dense_pm1(10, 1300)
    t = bf.autotune(dev(J), dev(h), 50)
    assert t["configs_per_s"] > 0
    en, st = bf.low_spectrum(dev(J), dev(h), 50)
    assert_int_equal(en.cpu().numpy(), bf.states_u64(st), *o.low_spectrum(J, h, 50))
