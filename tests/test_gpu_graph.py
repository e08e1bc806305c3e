"""bf_low_spectrum without host synchronisation: captured in a CUDA graph and replayed, with the
inputs changed in place between replays, and two searches queued on two streams at once (they
share the device's table of step increments, which the library orders between streams).
Every result is compared with the oracle."""
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


def compare(o, J, h, en, st, S):
    from paper_1904_03621_gb300 import api
    en = en.cpu().numpy()
    st = api.states_u64(st)
    if np.issubdtype(J.dtype, np.integer):
        assert_int_equal(en, st, *o.low_spectrum(J, h, S))
    else:
        assert_float_parity(o, J, h, en, st, *o.low_spectrum(J, h, S + 1))


@pytest.mark.parametrize("kind,n,S,kw", [("float", 24, 100, {}), ("int", 22, 300, {}),
                                         ("float", 26, 64, {"inner_bits": 10}),
                                         ("float", 30, 50, {"fixed_bits": 6, "fixed_value": 41}),
                                         ("float", 11, 20, {})])
def test_graph_capture_and_replay(bf, kind, n, S, kw):
    import torch
    from paper_1904_03621_gb300 import _lib
    o = oracle.get()
    make = instances.dense_gaussian if kind == "float" else instances.dense_pm1
    J, h = make(n, 700 + n)
    Jd = torch.from_numpy(np.ascontiguousarray(J)).cuda()
    hd = torch.from_numpy(np.ascontiguousarray(h)).cuda()
    ws = torch.empty(bf.workspace_size(n, S, Jd.dtype, **kw), dtype=torch.uint8, device="cuda")
    edt = torch.int64 if Jd.dtype == torch.int32 else torch.float64
    en = torch.empty(S, dtype=edt, device="cuda")
    st = torch.empty(S, dtype=torch.int64, device="cuda")
    bf.low_spectrum(Jd, hd, S, workspace=ws, out=(en, st), **kw)          # warm-up outside the capture
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bf.low_spectrum(Jd, hd, S, workspace=ws, out=(en, st), check=False, **kw)
    lib = _lib.load()
    Jo, ho = J, h
    fb, fv = kw.get("fixed_bits", 0), kw.get("fixed_value", 0)
    for rep in range(3):
        if rep == 2:                                  # a new instance written into the captured inputs
            Jo, ho = make(n, 800 + n)
            Jd.copy_(torch.from_numpy(np.ascontiguousarray(Jo)))
            hd.copy_(torch.from_numpy(np.ascontiguousarray(ho)))
        en.zero_()
        st.zero_()
        g.replay()
        torch.cuda.synchronize()
        _lib.check(lib.bf_workspace_status(ws.data_ptr(), None), lib)
        if fb:
            en_c, st_c = en.cpu().numpy(), bf.states_u64(st)
            en_o, st_o = o.low_spectrum(Jo, ho, S + 1, fixed_bits=fb, fixed_value=fv)
            assert_float_parity(o, Jo, ho, en_c, st_c, en_o, st_o)
        else:
            compare(o, Jo, ho, en, st, S)


def test_two_streams_at_once(bf):
    """Searches of two instances queued on two streams without synchronisation in between: the
    second search's walk must wait for the first one's before the shared increment table changes."""
    import torch
    o = oracle.get()
    cases = [instances.dense_gaussian(26, 901), instances.dense_pm1(25, 902), instances.dense_gaussian(24, 903)]
    streams = [torch.cuda.Stream() for _ in cases]
    outs = []
    torch.cuda.synchronize()
    for (J, h), s in zip(cases, streams):
        with torch.cuda.stream(s):
            Jd = torch.from_numpy(np.ascontiguousarray(J)).cuda()
            hd = torch.from_numpy(np.ascontiguousarray(h)).cuda()
            outs.append(bf.low_spectrum(Jd, hd, 200, stream=s, check=False) + (Jd, hd))
    torch.cuda.synchronize()
    for (J, h), (en, st, _, _) in zip(cases, outs):
        compare(o, J, h, en, st, 200)


@pytest.mark.parametrize("q,n,S", [(3, 10, 50), (4, 8, 30), (2, 16, 40)])
def test_potts_graph_capture_and_replay(bf, q, n, S):
    """The q-state Potts search (walk for q >= 3, the Ising map for q = 2) captured and replayed
    with new values written into the captured inputs."""
    import torch
    from paper_1904_03621_gb300 import _lib
    o = oracle.get()
    rng = np.random.default_rng(40 + q)

    def draw():
        J = np.triu(rng.standard_normal((n, n)), 1)
        return J + J.T, rng.standard_normal((n, q))
    J, h = draw()
    Jd = torch.from_numpy(np.ascontiguousarray(J)).cuda()
    hd = torch.from_numpy(np.ascontiguousarray(h)).cuda()
    lib = _lib.load()
    import ctypes
    o_ = bf._options()
    ws = torch.empty(int(lib.bf_potts_workspace_size(n, q, S, _lib.BF_F64, ctypes.byref(o_))), dtype=torch.uint8,
                     device="cuda")
    en = torch.empty(S, dtype=torch.float64, device="cuda")
    st = torch.empty(S, dtype=torch.int64, device="cuda")
    bf.low_spectrum_potts(Jd, hd, S, workspace=ws, out=(en, st))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bf.low_spectrum_potts(Jd, hd, S, workspace=ws, out=(en, st), check=False)
    for rep in range(2):
        if rep == 1:
            J, h = draw()
            Jd.copy_(torch.from_numpy(np.ascontiguousarray(J)))
            hd.copy_(torch.from_numpy(np.ascontiguousarray(h)))
        en.zero_()
        g.replay()
        torch.cuda.synchronize()
        _lib.check(lib.bf_workspace_status(ws.data_ptr(), None), lib)
        e_o, s_o = o.potts_low_spectrum(J, h, S)
        assert np.abs(en.cpu().numpy() - e_o).max() <= 1e-9 * (np.abs(np.triu(J, 1)).sum() + np.abs(h).sum())
        assert np.array_equal(bf.states_u64(st), s_o)
