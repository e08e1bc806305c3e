"""Cursor of the resumable search: host-side layout, validation and digest (CPU only)."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1904_03621_gb300 import _lib
from paper_1904_03621_gb300.checkpoint import instance_digest


@pytest.fixture(scope="module")
def lib():
    from paper_1904_03621_gb300 import build
    build.build()
    return _lib.load()


def make(lib, n=20, S=16, dtype=_lib.BF_I32, chunk_bits=3, digest=123):
    nbytes = lib.bf_cursor_bytes(S)
    buf = ctypes.create_string_buffer(nbytes)
    st = lib.bf_cursor_init(buf, nbytes, n, S, dtype, chunk_bits, digest)
    return st, buf, nbytes


def state(lib, buf, nbytes):
    nxt, tot, cnt = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
    st = lib.bf_cursor_state(buf, nbytes, ctypes.byref(nxt), ctypes.byref(tot), None, None, ctypes.byref(cnt))
    return st, nxt.value, tot.value, cnt.value


def test_layout_and_fresh_state(lib):
    assert lib.bf_cursor_bytes(16) == 128 + 16 * 16
    assert lib.bf_cursor_bytes(0) == 0 and lib.bf_cursor_bytes(4096) == 0
    st, buf, nbytes = make(lib, chunk_bits=5)
    assert st == _lib.BF_OK
    assert buf.raw[:8] == b"BFCURSR1"
    assert state(lib, buf, nbytes) == (_lib.BF_OK, 0, 32, 0)


def test_init_rejects_bad_arguments(lib):
    assert make(lib, n=10, S=16, chunk_bits=7)[0] == _lib.BF_EINVAL      # 2^3 configurations < S
    assert make(lib, n=10, chunk_bits=11)[0] == _lib.BF_EINVAL           # chunk_bits > n
    assert make(lib, n=65)[0] == _lib.BF_EINVAL
    assert make(lib, dtype=7)[0] == _lib.BF_EINVAL
    nbytes = lib.bf_cursor_bytes(16)
    small = ctypes.create_string_buffer(nbytes - 1)
    assert lib.bf_cursor_init(small, nbytes - 1, 20, 16, 0, 3, 1) == _lib.BF_EINVAL


def test_corruption_is_detected(lib):
    st, buf, nbytes = make(lib)
    raw = bytearray(buf.raw)
    for pos in (3, 40, 200):                     # magic, header field, record area
        bad = bytearray(raw)
        bad[pos] ^= 0x10
        b2 = ctypes.create_string_buffer(bytes(bad), nbytes)
        assert state(lib, b2, nbytes)[0] == _lib.BF_EINVAL, pos
    # a future version is refused as unsupported, not misread
    bad = bytearray(raw)
    bad[8] = 2
    b2 = ctypes.create_string_buffer(bytes(bad), nbytes)
    assert state(lib, b2, nbytes)[0] in (_lib.BF_EINVAL, _lib.BF_EUNSUPPORTED)
    assert state(lib, buf, nbytes - 1)[0] == _lib.BF_EINVAL       # truncated buffer


def test_digest_reads_the_upper_triangle_and_fields(lib):
    rng = np.random.default_rng(0)
    J = rng.standard_normal((9, 9))
    h = rng.standard_normal(9)
    d = instance_digest(J, h, _lib.BF_F64)
    J2 = J.copy()
    J2[np.tril_indices(9)] = 7.0                   # diagonal and lower triangle are not read
    assert instance_digest(J2, h, _lib.BF_F64) == d
    J3 = J.copy()
    J3[2, 5] += 1e-12
    assert instance_digest(J3, h, _lib.BF_F64) != d
    h2 = h.copy()
    h2[8] = -h2[8]
    assert instance_digest(J, h2, _lib.BF_F64) != d
    assert instance_digest(J, h, _lib.BF_F32) != d
