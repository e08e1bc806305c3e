"""q-state Potts model (the extension to other classical spin-glass models named in
Sec. 2) on the GPU against the oracle's Potts energy by definition."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from parity import assert_float_parity, assert_int_equal

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


def potts_instance(n, q, seed, integer=True):
    rng = np.random.default_rng(seed)
    if integer:
        J = rng.integers(-7, 8, (n, n)).astype(np.int32)
        h = rng.integers(-7, 8, (n, q)).astype(np.int32)
    else:
        J = rng.standard_normal((n, n))
        h = rng.standard_normal((n, q))
    return J, h


def run(bf, J, h, S, **kw):
    import torch
    e, st = bf.low_spectrum_potts(torch.as_tensor(np.ascontiguousarray(J)).cuda(),
                                  torch.as_tensor(np.ascontiguousarray(h)).cuda(), S, **kw)
    return e.cpu().numpy(), bf.states_u64(st)


@pytest.mark.parametrize("q,n,S,seed", [(2, 20, 100, 0), (3, 14, 100, 1), (4, 11, 300, 2), (5, 9, 50, 3),
                                        (6, 8, 64, 4), (7, 7, 1000, 5), (8, 7, 77, 6), (3, 16, 2048, 7)])
def test_potts_int_exact(bf, o, q, n, S, seed):
    J, h = potts_instance(n, q, seed)
    e, st = run(bf, J, h, S)
    e_o, st_o = o.potts_low_spectrum(J, h, S)
    assert_int_equal(e, st, e_o, st_o)


@pytest.mark.parametrize("q,n,S", [(3, 5, 243), (8, 4, 100), (2, 12, 10), (4, 6, 2048)])
def test_potts_direct_path(bf, o, q, n, S):
    J, h = potts_instance(n, q, 10 + q)
    e, st = run(bf, J, h, S)
    e_o, st_o = o.potts_low_spectrum(J, h, S)
    assert_int_equal(e, st, e_o, st_o)


@pytest.mark.parametrize("q,n,S", [(3, 13, 60), (4, 10, 40), (2, 22, 60)])
def test_potts_float(bf, o, q, n, S):
    import torch
    J, h = potts_instance(n, q, 20 + q, integer=False)
    e, st = run(bf, J, h, S)
    e_o, st_o = o.potts_low_spectrum(J, h, S + 1)
    assert_float_parity(o, J, h, e, st, e_o, st_o, energy=o.potts_energy)
    J32, h32 = J.astype(np.float32), h.astype(np.float32)
    e, st = run(bf, J32, h32, S)
    e_o, st_o = o.potts_low_spectrum(J32.astype(np.float64), h32.astype(np.float64), S + 1)
    assert_float_parity(o, J32.astype(np.float64), h32.astype(np.float64), e, st, e_o, st_o, energy=o.potts_energy)


def test_potts_q2_matches_ising_entry(bf):
    """q = 2 through the Potts path equals the Ising path on J/2, (h1 - h0)/2 up to a constant."""
    import torch
    rng = np.random.default_rng(40)
    n = 22
    K = rng.integers(-5, 6, (n, n)).astype(np.int32)
    J = 2 * K
    h0 = rng.integers(-5, 6, n).astype(np.int32)
    h = np.stack([h0, h0 + 2 * rng.integers(-5, 6, n)], axis=1).astype(np.int32)
    e_p, st_p = run(bf, J, h, 200)
    e_i, st_i = bf.low_spectrum(torch.tensor(K).cuda(), torch.tensor((h[:, 1] - h[:, 0]) // 2).cuda(), 200)
    const = int(np.triu(K, 1).sum()) + int(h.sum()) // 2
    assert np.array_equal(st_p, bf.states_u64(st_i))
    assert np.array_equal(e_p, e_i.cpu().numpy() + const)


def test_potts_task_sizes_agree(bf, o):
    J, h = potts_instance(15, 3, 50)
    ref = None
    for kw in ({}, {"grid_blocks": 3}, {"grid_blocks": 1}):
        e, st = run(bf, J, h, 500, **kw)
        if ref is None:
            ref = (e, st)
            e_o, st_o = o.potts_low_spectrum(J, h, 500)
            assert_int_equal(e, st, e_o, st_o)
        else:
            assert_int_equal(e, st, *ref)


def test_potts_errors(bf):
    import torch
    from paper_1904_03621_gb300 import _lib
    J = torch.zeros((5, 5), dtype=torch.int32).cuda()
    with pytest.raises(_lib.BFError) as err:
        bf.low_spectrum_potts(J, torch.zeros((5, 9), dtype=torch.int32).cuda(), 4)   # q = 9
    assert err.value.status == _lib.BF_EUNSUPPORTED
    with pytest.raises(_lib.BFError) as err:
        bf.low_spectrum_potts(J, torch.zeros((5, 3), dtype=torch.int32).cuda(), 244)  # S > 3^5
    assert err.value.status == _lib.BF_EINVAL
    with pytest.raises(ValueError):
        bf.low_spectrum_potts(J, torch.zeros(5, dtype=torch.int32).cuda(), 4)
