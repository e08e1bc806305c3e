"""QUBO form (Sec. 2, Eqs. (2)-(3)) and the dict-graph front end on the GPU, against
the oracle's QUBO value by definition."""
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


def qubo_instance(n, seed, integer, scale=9):
    """Coefficients with junk on the diagonal and lower triangle (must be ignored)."""
    rng = np.random.default_rng(seed)
    if integer:
        return (rng.integers(-scale, scale + 1, (n, n)).astype(np.int32),
                rng.integers(-scale, scale + 1, n).astype(np.int32))
    return rng.standard_normal((n, n)), rng.standard_normal(n)


def run(bf, a, b, S, torch_dtype=None, **kw):
    import torch
    at = torch.as_tensor(np.ascontiguousarray(a))
    bt = torch.as_tensor(np.ascontiguousarray(b))
    if torch_dtype is not None:
        at, bt = at.to(torch_dtype), bt.to(torch_dtype)
    F, st = bf.low_spectrum_qubo(at.cuda(), bt.cuda(), S, **kw)
    return F.cpu().numpy(), bf.states_u64(st)


@pytest.mark.parametrize("n,S,seed", [(5, 32, 0), (12, 100, 1), (20, 1000, 2), (26, 64, 3), (33, 10, 4)])
def test_qubo_int_exact(bf, o, n, S, seed):
    a, b = qubo_instance(n, seed, integer=True)
    kw = {"fixed_bits": n - 26, "fixed_value": 5} if n > 26 else {}
    F, st = run(bf, a, b, S, **kw)
    F_o, st_o = o.qubo_low_spectrum(a, b, S, **kw)
    assert_int_equal(F, st, F_o, st_o)


@pytest.mark.parametrize("n,S,seed", [(14, 50, 5), (22, 300, 6)])
def test_qubo_float(bf, o, n, S, seed):
    import torch
    a, b = qubo_instance(n, seed, integer=False)
    for dt in (torch.float64, torch.float32):
        a_in = a.astype(np.float32).astype(np.float64) if dt == torch.float32 else a
        b_in = b.astype(np.float32).astype(np.float64) if dt == torch.float32 else b
        F, st = run(bf, a_in, b_in, S, torch_dtype=dt)
        F_o, st_o = o.qubo_low_spectrum(a_in, b_in, S + 1)
        assert_float_parity(o, a_in, b_in, F, st, F_o, st_o, energy=o.qubo_energy)


def test_qubo_tensor_core_variant(bf, o):
    a, b = qubo_instance(20, 7, integer=True)
    F, st = run(bf, a, b, 200, variant=2)
    F_o, st_o = o.qubo_low_spectrum(a, b, 200)
    assert_int_equal(F, st, F_o, st_o)


def test_qubo_int_range_error(bf):
    import torch
    from paper_1904_03621_gb300 import _lib
    n = 4
    a = np.full((n, n), 2**30, dtype=np.int32)
    b = np.zeros(n, dtype=np.int32)
    with pytest.raises(_lib.BFError) as err:
        bf.low_spectrum_qubo(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), 4)
    assert err.value.status == _lib.BF_EUNSUPPORTED


def test_search_paper_example(bf):
    """The paper's usage example (Sec. 4.1): nodes 1, 2; (1,1) -> field, (1,2) -> coupling."""
    from paper_1904_03621_gb300 import search
    sol = search({(1, 1): -1, (1, 2): -0.2}, num_states=4)
    # E = -0.2 s1 s2 - s1 (library sign): (s1, s2) = (+,+) -1.2, (+,-) -0.8, (-,-) 0.8, (-,+) 1.2
    assert np.allclose(sol.energies, [-1.2, -0.8, 0.8, 1.2])
    assert [tuple(r) for r in sol.states] == [(1, 1), (1, -1), (-1, -1), (-1, 1)]
    assert sol.nodes == [1, 2]
    assert list(sol.configurations) == [3, 1, 0, 2]


def test_search_dict_graph(bf, o):
    """A sparse dict graph with string labels against the oracle on the dense form."""
    from paper_1904_03621_gb300 import search
    from paper_1904_03621_gb300.graph import graph_to_dense
    rng = np.random.default_rng(9)
    labels = [f"v{k:02d}" for k in range(18)]
    graph = {}
    for i in range(18):
        graph[(labels[i], labels[i])] = int(rng.integers(-3, 4))
        for j in rng.choice(18, 4, replace=False):
            if j != i:
                graph[(labels[i], labels[int(j)])] = int(rng.integers(-3, 4))
    for qubo in (False, True):
        sol = search(graph, 50, qubo=qubo)
        J, h, nodes = graph_to_dense(graph)
        if qubo:
            e_o, st_o = o.qubo_low_spectrum(J, h, 50)
        else:
            e_o, st_o = o.low_spectrum(J, h, 50)
        assert_int_equal(sol.energies, sol.configurations, e_o, st_o)
        bits = ((st_o[:, None] >> np.arange(18, dtype=np.uint64)) & np.uint64(1)).astype(np.int8)
        assert np.array_equal(sol.states, bits if qubo else 2 * bits - 1)
