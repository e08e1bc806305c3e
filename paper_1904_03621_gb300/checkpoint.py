"""Checkpoint / restart of long exhaustive searches (the chunk loop of Algorithm 1).

`ResumableSearch` drives the library's cursor (`bf_cursor_*`, include/bf.h): the
space of 2^n configurations is split into 2^chunk_bits chunks (the top chunk_bits
bits of c fixed, Sec. 3, Eq. (6)); after every chunk the cursor -- next chunk and the
S lowest records so far -- is a self-contained byte string that `save` writes
atomically and `load` reads back.  The cursor checks that it is resumed on the same
instance (digest of J's upper triangle and h) and detects corrupted files (checksum).
This module only moves bytes between the library, torch and files.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _lib

_NP_OF = {_lib.BF_I32: np.int32, _lib.BF_F32: np.float32, _lib.BF_F64: np.float64}


def instance_digest(J: np.ndarray, h: np.ndarray, dtype: int) -> int:
    lib = _lib.load()
    J = np.ascontiguousarray(J, dtype=_NP_OF[dtype])
    h = np.ascontiguousarray(h, dtype=_NP_OF[dtype])
    return int(lib.bf_instance_digest(J.ctypes.data, h.ctypes.data, J.shape[0], dtype))


class ResumableSearch:
    """The S lowest (energy, configuration) pairs of one instance, computed chunk by chunk.

    J, h: CUDA tensors as for `api.low_spectrum`.  chunk_bits: log2 of the number of
    chunks.  cursor: bytes of a saved cursor to resume from (default: a new search).
    Other keyword options go to every chunk's search (variant, task_log2, ...).
    """

    def __init__(self, J, h, S: int, chunk_bits: int, cursor: bytes | None = None, **opts):
        import torch

        from . import api
        self._api = api
        self.lib = _lib.load()
        if J.dtype not in api._DTYPES or h.dtype != J.dtype:
            raise TypeError("J and h must share one of int32, float32, float64")
        self.J, self.h = J.contiguous(), h.contiguous()
        self.dtype = api._DTYPES[J.dtype]
        self.S = S
        self.opts = opts
        nbytes = self.lib.bf_cursor_bytes(S)
        if nbytes == 0:
            raise _lib.BFError(_lib.BF_EUNSUPPORTED, f"S={S} outside [1, BF_MAX_S]")
        self.buf = ctypes.create_string_buffer(nbytes)
        if cursor is None:
            digest = instance_digest(self.J.cpu().numpy(), self.h.cpu().numpy(), self.dtype)
            _lib.check(self.lib.bf_cursor_init(self.buf, nbytes, J.shape[0], S, self.dtype, chunk_bits, digest),
                       self.lib)
        else:
            if len(cursor) != nbytes:
                raise _lib.BFError(_lib.BF_EINVAL, f"cursor of {len(cursor)} bytes, expected {nbytes} for S={S}")
            ctypes.memmove(self.buf, cursor, nbytes)
        self.progress()   # validates the buffer (magic, version, checksum)
        o = api._options(**opts)
        ws = self.lib.bf_cursor_workspace_size(self.buf, nbytes, ctypes.byref(o))
        if ws == 0:
            raise _lib.BFError(_lib.BF_EINVAL, "options rejected for this cursor")
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=J.device)

    @classmethod
    def load(cls, path: str, J, h, S: int, **opts) -> "ResumableSearch":
        with open(path, "rb") as f:
            data = f.read()
        return cls(J, h, S, 0, cursor=data, **opts)

    def cursor(self) -> bytes:
        return self.buf.raw

    def save(self, path: str) -> None:
        """Write the cursor atomically (temporary file, fsync, rename)."""
        tmp = f"{path}.tmp.{os.getpid()}"
        with open(tmp, "wb") as f:
            f.write(self.buf.raw)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)

    def progress(self) -> tuple[int, int]:
        nxt, tot = ctypes.c_uint64(0), ctypes.c_uint64(0)
        _lib.check(self.lib.bf_cursor_state(self.buf, len(self.buf.raw), ctypes.byref(nxt), ctypes.byref(tot),
                                            None, None, None), self.lib)
        return int(nxt.value), int(tot.value)

    @property
    def done(self) -> bool:
        nxt, tot = self.progress()
        return nxt >= tot

    def step(self, max_chunks: int = 1, stream=None) -> bool:
        """Search up to max_chunks more chunks; returns True when the search is complete."""
        o = self._api._options(**self.opts)
        st = self.lib.bf_cursor_step(self.buf, len(self.buf.raw), self.J.data_ptr(), self.h.data_ptr(),
                                     int(max_chunks), self.workspace.data_ptr(), self.workspace.numel(),
                                     ctypes.byref(o), self._api._stream_handle(stream))
        _lib.check(st, self.lib)
        return self.done

    def run(self, checkpoint_path: str | None = None, chunks_per_save: int = 1) -> None:
        while not self.done:
            self.step(chunks_per_save)
            if checkpoint_path:
                self.save(checkpoint_path)

    def result(self):
        """(energies, states) of the records so far: int64 or float64, uint64; ascending by (E, c)."""
        S = self.S
        en = np.empty(S, dtype=np.int64 if self.dtype == _lib.BF_I32 else np.float64)
        st = np.empty(S, dtype=np.uint64)
        cnt = ctypes.c_int(0)
        _lib.check(self.lib.bf_cursor_state(self.buf, len(self.buf.raw), None, None, en.ctypes.data,
                                            st.ctypes.data, ctypes.byref(cnt)), self.lib)
        return en[:cnt.value], st[:cnt.value]
