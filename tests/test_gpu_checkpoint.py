"""Checkpoint / restart of the chunked search on the GPU: results identical to the
single-call search and to the oracle; resume across processes' worth of save/load."""
from __future__ import annotations

import os

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


@pytest.fixture(scope="module")
def o():
    return oracle.get()


def test_resume_chunk_by_chunk_int(bf, o, tmp_path):
    import torch
    from paper_1904_03621_gb300.checkpoint import ResumableSearch
    J, h = instances.dense_pm1(26, 31)
    Jt, ht = torch.tensor(J).cuda(), torch.tensor(h).cuda()
    S = 100
    path = os.path.join(tmp_path, "search.cursor")
    rs = ResumableSearch(Jt, ht, S, chunk_bits=3)
    rs.step(1)
    rs.save(path)
    del rs
    steps = 1
    while True:                                   # a fresh object per chunk, as after a restart
        rs = ResumableSearch.load(path, Jt, ht, S)
        if rs.done:
            break
        rs.step(1)
        rs.save(path)
        steps += 1
    assert steps == 8 and rs.progress() == (8, 8)
    en, st = rs.result()
    en_full, st_full = bf.low_spectrum(Jt, ht, S)
    assert_int_equal(en, st, en_full.cpu().numpy(), bf.states_u64(st_full))
    en_o, st_o = o.low_spectrum(J, h, S)
    assert_int_equal(en, st, en_o, st_o)


def test_resume_float_equals_single_call(bf, o):
    import torch
    from paper_1904_03621_gb300.checkpoint import ResumableSearch
    J, h = instances.dense_gaussian(24, 32)
    Jt, ht = torch.tensor(J).cuda(), torch.tensor(h).cuda()
    S = 50
    rs = ResumableSearch(Jt, ht, S, chunk_bits=2)
    rs.step(3)
    assert rs.progress() == (3, 4)
    rs2 = ResumableSearch(Jt, ht, S, 0, cursor=rs.cursor())
    rs2.run()
    en, st = rs2.result()
    en_full, st_full = bf.low_spectrum(Jt, ht, S)
    assert np.array_equal(en, en_full.cpu().numpy()) and np.array_equal(st, bf.states_u64(st_full))
    en_o, st_o = o.low_spectrum(J, h, S + 1)
    assert_float_parity(o, J, h, en, st, en_o, st_o)


def test_partial_list_is_a_lower_bound(bf, o):
    """After k of 2^c chunks the list is the exact top-S of those chunks' union."""
    import torch
    from paper_1904_03621_gb300.checkpoint import ResumableSearch
    J, h = instances.dense_pm1(22, 33)
    Jt, ht = torch.tensor(J).cuda(), torch.tensor(h).cuda()
    rs = ResumableSearch(Jt, ht, 40, chunk_bits=2, variant=2)
    rs.step(2)                                    # chunks 0 and 1: top bit of c is 0
    en, st = rs.result()
    en_o, st_o = o.low_spectrum(J, h, 40, fixed_bits=1, fixed_value=0)
    assert_int_equal(en, st, en_o, st_o)


def test_cursor_refuses_other_instance_and_corruption(bf, tmp_path):
    import torch
    from paper_1904_03621_gb300 import _lib
    from paper_1904_03621_gb300.checkpoint import ResumableSearch
    J, h = instances.dense_pm1(20, 34)
    Jt, ht = torch.tensor(J).cuda(), torch.tensor(h).cuda()
    rs = ResumableSearch(Jt, ht, 10, chunk_bits=2)
    rs.step(1)
    J2 = J.copy()
    J2[0, 1] = -J2[0, 1]
    other = ResumableSearch(torch.tensor(J2).cuda(), ht, 10, 0, cursor=rs.cursor())
    with pytest.raises(_lib.BFError) as err:
        other.step(1)
    assert err.value.status == _lib.BF_EINVAL
    bad = bytearray(rs.cursor())
    bad[130] ^= 1
    with pytest.raises(_lib.BFError):
        ResumableSearch(Jt, ht, 10, 0, cursor=bytes(bad))
