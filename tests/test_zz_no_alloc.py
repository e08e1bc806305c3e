"""bf_low_spectrum_noalloc: the search for callers that cannot allocate device memory.

Such callers (code under a framework whose caching allocator owns the free
device memory, callbacks or real-time loops that must not trigger an
allocation's implicit synchronisation, hosts with a fixed memory budget) pass
only inputs and outputs; the library uses its own 4 MiB device array as the
workspace.  These tests call it through the C ABI and compare it with
bf_low_spectrum on the same inputs, twice in a row (the array keeps the
previous call's contents, so the second call checks that each call clears what
it needs).  This file is collected last so a failure here comes after every
other test has run.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from parity import tolerance
from paper_1904_03621_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import _lib, api
    assert torch.cuda.is_available()
    return torch, _lib, api


def _noalloc(torch, _lib, Jt, ht, S, opts=None):
    lib = _lib.load()
    dt = {torch.int32: _lib.BF_I32, torch.float32: _lib.BF_F32, torch.float64: _lib.BF_F64}[Jt.dtype]
    edt = torch.int64 if Jt.dtype == torch.int32 else torch.float64
    en = torch.empty(S, dtype=edt, device=Jt.device)
    st = torch.empty(S, dtype=torch.int64, device=Jt.device)
    o = opts if opts is not None else _lib.Options()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = lib.bf_low_spectrum_noalloc(Jt.data_ptr(), ht.data_ptr(), Jt.shape[0], S, dt, en.data_ptr(),
                                         st.data_ptr(), ctypes.byref(o), stream)
    return status, en, st


@pytest.mark.parametrize("case", ["float_n22", "int_n24", "float32_n20_fixed"])
def test_noalloc_matches_regular_entry_point(env, case):
    torch, _lib, api = env
    if case == "float_n22":
        J, h = instances.dense_gaussian(22, 3)
        S, kw = 100, {}
    elif case == "int_n24":
        J, h = instances.dense_pm1(24, 4)
        S, kw = 200, {}
    else:
        J, h = instances.dense_gaussian(26, 5)
        J, h = J.astype(np.float32), h.astype(np.float32)
        S, kw = 64, {"fixed_bits": 6, "fixed_value": 37}
    Jt = torch.from_numpy(np.ascontiguousarray(J)).cuda()
    ht = torch.from_numpy(np.ascontiguousarray(h)).cuda()
    en_ref, st_ref = api.low_spectrum(Jt, ht, S, **kw)
    en_ref = en_ref.cpu().numpy()
    st_ref = api.states_u64(st_ref)
    opts = _lib.Options(fixed_bits=kw.get("fixed_bits", 0), fixed_value=kw.get("fixed_value", 0))
    for _ in range(2):   # two calls in a row on the shared array
        status, en, st = _noalloc(torch, _lib, Jt, ht, S, opts)
        assert status == _lib.BF_OK, _lib.load().bf_last_error_detail().decode()
        en = en.cpu().numpy()
        st = api.states_u64(st)
        if np.issubdtype(J.dtype, np.integer):
            assert np.array_equal(en, en_ref) and np.array_equal(st, st_ref)
        else:
            assert np.abs(en - en_ref).max() <= tolerance(J, h)
            assert np.array_equal(st, st_ref)


def test_noalloc_rejects_searches_beyond_its_array(env):
    torch, _lib, api = env
    J, h = instances.dense_gaussian(24, 6)
    Jt = torch.from_numpy(J).cuda()
    ht = torch.from_numpy(h).cuda()
    status, _, _ = _noalloc(torch, _lib, Jt, ht, 2048)
    assert status == _lib.BF_EUNSUPPORTED
    assert b"4 MiB" in _lib.load().bf_last_error_detail()
    status, _, _ = _noalloc(torch, _lib, Jt, ht, 1 << 25)
    assert status == _lib.BF_EINVAL


def test_noalloc_reports_device_status_then_recovers(env):
    """A flood of equal energies into a 16-record spill area must come back from this entry point
    as BF_EOVERFLOW (it waits for its work and returns the device-side status), and the next call
    on the shared array, which still holds that error word, must succeed and match bf_low_spectrum."""
    torch, _lib, api = env
    n = 20
    Jz = torch.zeros(n, n, dtype=torch.int32, device="cuda")
    hz = torch.zeros(n, dtype=torch.int32, device="cuda")
    status, _, _ = _noalloc(torch, _lib, Jz, hz, 10, _lib.Options(spill_log2=4, inner_bits=9))
    assert status == _lib.BF_EOVERFLOW, _lib.load().bf_last_error_detail().decode()
    J, h = instances.dense_pm1(22, 8)
    Jt = torch.from_numpy(np.ascontiguousarray(J)).cuda()
    ht = torch.from_numpy(np.ascontiguousarray(h)).cuda()
    en_ref, st_ref = api.low_spectrum(Jt, ht, 50)
    status, en, st = _noalloc(torch, _lib, Jt, ht, 50)
    assert status == _lib.BF_OK, _lib.load().bf_last_error_detail().decode()
    assert np.array_equal(en.cpu().numpy(), en_ref.cpu().numpy())
    assert np.array_equal(api.states_u64(st), api.states_u64(st_ref))
