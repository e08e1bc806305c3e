"""Oracle: exhaustive CPU enumeration of the S lowest Ising states.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_1904_03621_gb300``) and neither
imports the other.

The arithmetic lives in ``oracle.c`` (plain C + OpenMP, FP64 / int64, direct
definition of Eq. (1) of the paper, Sec. 2, with the library's sign and
encoding conventions).  This module only compiles it with gcc and marshals
numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DEFAULT = os.path.join(_HERE, "liboracle.so")


def build(out_path: str | None = None, plant: int = 0, quiet: bool = True) -> str:
    """Compile oracle.c into a shared library and return its path.

    ``plant`` > 0 compiles a copy with one deliberate mistake (see the
    ORACLE_PLANT switch in oracle.c); such copies go to a temporary
    directory and are used only by the mutation tests.
    """
    if out_path is None:
        if plant:
            out_path = os.path.join(tempfile.mkdtemp(prefix="oracle_plant_"), f"liboracle_p{plant}.so")
        else:
            out_path = _LIB_DEFAULT
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           f"-DORACLE_PLANT={int(plant)}", _SRC, "-o", out_path]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + res.stderr)
    if not quiet and res.stderr:
        print(res.stderr)
    return out_path


class Oracle:
    """ctypes handle on one compiled copy of oracle.c."""

    def __init__(self, path: str | None = None):
        if path is None:
            path = _LIB_DEFAULT
            if (not os.path.exists(path)) or os.path.getmtime(path) < os.path.getmtime(_SRC):
                build(path)
        self.path = path
        lib = ctypes.CDLL(path)
        u64, i64, i32, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        vp = ctypes.c_void_p
        lib.oracle_energy_f64.restype = dbl
        lib.oracle_energy_f64.argtypes = [i32, vp, vp, u64]
        lib.oracle_energy_i64.restype = i64
        lib.oracle_energy_i64.argtypes = [i32, vp, vp, u64]
        lib.oracle_potts_energy_f64.restype = dbl
        lib.oracle_potts_energy_f64.argtypes = [i32, i32, vp, vp, u64]
        lib.oracle_potts_energy_i64.restype = i64
        lib.oracle_potts_energy_i64.argtypes = [i32, i32, vp, vp, u64]
        for name in ("oracle_potts_low_spectrum_f64", "oracle_potts_low_spectrum_i64"):
            f = getattr(lib, name)
            f.restype = i32
            f.argtypes = [i32, i32, vp, vp, i32, i32, i32, vp, vp]
        lib.oracle_qubo_energy_f64.restype = dbl
        lib.oracle_qubo_energy_f64.argtypes = [i32, vp, vp, u64]
        lib.oracle_qubo_energy_i64.restype = i64
        lib.oracle_qubo_energy_i64.argtypes = [i32, vp, vp, u64]
        for name in ("oracle_low_spectrum_f64", "oracle_low_spectrum_i64", "oracle_qubo_low_spectrum_f64",
                     "oracle_qubo_low_spectrum_i64"):
            f = getattr(lib, name)
            f.restype = i32
            f.argtypes = [i32, vp, vp, i32, i32, u64, i32, i32, vp, vp]
        lib.oracle_all_energies_f64.restype = i32
        lib.oracle_all_energies_f64.argtypes = [i32, vp, vp, vp]
        lib.oracle_all_energies_i64.restype = i32
        lib.oracle_all_energies_i64.argtypes = [i32, vp, vp, vp]
        lib.oracle_grad.restype = i32
        lib.oracle_grad.argtypes = [i32, vp, i32, vp, vp, vp, vp, vp, vp]
        lib.oracle_num_threads.restype = i32
        lib.oracle_plant.restype = i32
        self.lib = lib

    # -- helpers -------------------------------------------------------
    @staticmethod
    def _is_int(J) -> bool:
        return np.issubdtype(np.asarray(J).dtype, np.integer)

    @staticmethod
    def _prep(J, h):
        J = np.asarray(J)
        h = np.asarray(h)
        n = J.shape[0]
        assert J.shape == (n, n) and h.shape == (n,)
        if np.issubdtype(J.dtype, np.integer):
            return n, np.ascontiguousarray(J, dtype=np.int32), np.ascontiguousarray(h, dtype=np.int32)
        return n, np.ascontiguousarray(J, dtype=np.float64), np.ascontiguousarray(h, dtype=np.float64)

    @property
    def num_threads(self) -> int:
        return int(self.lib.oracle_num_threads())

    # -- Eq. (1) ---------------------------------------------------------
    def energy(self, J, h, c: int):
        n, J, h = self._prep(J, h)
        if self._is_int(J):
            return int(self.lib.oracle_energy_i64(n, J.ctypes.data, h.ctypes.data, int(c)))
        return float(self.lib.oracle_energy_f64(n, J.ctypes.data, h.ctypes.data, int(c)))

    def all_energies(self, J, h) -> np.ndarray:
        n, J, h = self._prep(J, h)
        if self._is_int(J):
            out = np.empty(1 << n, dtype=np.int64)
            rc = self.lib.oracle_all_energies_i64(n, J.ctypes.data, h.ctypes.data, out.ctypes.data)
        else:
            out = np.empty(1 << n, dtype=np.float64)
            rc = self.lib.oracle_all_energies_f64(n, J.ctypes.data, h.ctypes.data, out.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle_all_energies failed rc={rc}")
        return out

    # -- Algorithm 1 contract ----------------------------------------------
    def low_spectrum(self, J, h, S: int, fixed_bits: int = 0, fixed_value: int = 0,
                     mode: int = 0, threads: int = 0):
        """S lowest (energy, state) pairs, ordered by (E, c).

        Returns (energies, states): int64 energies for integer instances,
        float64 otherwise; states are uint64 configuration integers.
        """
        n, J, h = self._prep(J, h)
        states = np.empty(S, dtype=np.uint64)
        if self._is_int(J):
            en = np.empty(S, dtype=np.int64)
            f = self.lib.oracle_low_spectrum_i64
        else:
            en = np.empty(S, dtype=np.float64)
            f = self.lib.oracle_low_spectrum_f64
        rc = f(n, J.ctypes.data, h.ctypes.data, int(S), int(fixed_bits), int(fixed_value),
               int(mode), int(threads), en.ctypes.data, states.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle_low_spectrum failed rc={rc}")
        return en, states

    # -- QUBO form, Eq. (2) with the library's sign ---------------------------
    def qubo_energy(self, a, b, c: int):
        n, a, b = self._prep(a, b)
        if self._is_int(a):
            return int(self.lib.oracle_qubo_energy_i64(n, a.ctypes.data, b.ctypes.data, int(c)))
        return float(self.lib.oracle_qubo_energy_f64(n, a.ctypes.data, b.ctypes.data, int(c)))

    def qubo_low_spectrum(self, a, b, S: int, fixed_bits: int = 0, fixed_value: int = 0,
                          mode: int = 0, threads: int = 0):
        """S lowest (F, c) pairs of F(q) = sum_{i<j} a_ij q_i q_j + sum_i b_i q_i, by (F, c)."""
        n, a, b = self._prep(a, b)
        states = np.empty(S, dtype=np.uint64)
        if self._is_int(a):
            val = np.empty(S, dtype=np.int64)
            f = self.lib.oracle_qubo_low_spectrum_i64
        else:
            val = np.empty(S, dtype=np.float64)
            f = self.lib.oracle_qubo_low_spectrum_f64
        rc = f(n, a.ctypes.data, b.ctypes.data, int(S), int(fixed_bits), int(fixed_value),
               int(mode), int(threads), val.ctypes.data, states.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle_qubo_low_spectrum failed rc={rc}")
        return val, states

    # -- q-state Potts model ------------------------------------------------------
    @staticmethod
    def _prep_potts(J, h):
        J = np.asarray(J)
        h = np.asarray(h)
        n, q = h.shape
        assert J.shape == (n, n)
        dt = np.int32 if np.issubdtype(J.dtype, np.integer) else np.float64
        return n, q, np.ascontiguousarray(J, dtype=dt), np.ascontiguousarray(h, dtype=dt)

    def potts_energy(self, J, h, c: int):
        """E = sum_{i<j} J_ij [sigma_i == sigma_j] + sum_i h[i, sigma_i], sigma_i = base-q digit i of c."""
        n, q, J, h = self._prep_potts(J, h)
        if self._is_int(J):
            return int(self.lib.oracle_potts_energy_i64(n, q, J.ctypes.data, h.ctypes.data, int(c)))
        return float(self.lib.oracle_potts_energy_f64(n, q, J.ctypes.data, h.ctypes.data, int(c)))

    def potts_low_spectrum(self, J, h, S: int, mode: int = 0, threads: int = 0):
        """S lowest (E, c) of the Potts model (h of shape (n, q)), ordered by (E, c)."""
        n, q, J, h = self._prep_potts(J, h)
        states = np.empty(S, dtype=np.uint64)
        if self._is_int(J):
            en = np.empty(S, dtype=np.int64)
            f = self.lib.oracle_potts_low_spectrum_i64
        else:
            en = np.empty(S, dtype=np.float64)
            f = self.lib.oracle_potts_low_spectrum_f64
        rc = f(n, q, J.ctypes.data, h.ctypes.data, int(S), int(mode), int(threads), en.ctypes.data,
               states.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle_potts_low_spectrum failed rc={rc}")
        return en, states

    # -- gradient of sum_k g_k E_k (linearity of Eq. (1)) --------------------
    def grad(self, n_list, states, g):
        n_arr = np.ascontiguousarray(n_list, dtype=np.int32)
        B = n_arr.shape[0]
        states = np.ascontiguousarray(states, dtype=np.uint64).reshape(B, -1)
        S = states.shape[1]
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(B, S)
        J_off = np.zeros(B, dtype=np.int64)
        h_off = np.zeros(B, dtype=np.int64)
        J_off[1:] = np.cumsum(n_arr.astype(np.int64) ** 2)[:-1]
        h_off[1:] = np.cumsum(n_arr.astype(np.int64))[:-1]
        dJ = np.zeros(int((n_arr.astype(np.int64) ** 2).sum()), dtype=np.float64)
        dh = np.zeros(int(n_arr.sum()), dtype=np.float64)
        rc = self.lib.oracle_grad(B, n_arr.ctypes.data, S, states.ctypes.data, g.ctypes.data,
                                  J_off.ctypes.data, h_off.ctypes.data, dJ.ctypes.data, dh.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle_grad failed rc={rc}")
        return dJ, dh, J_off, h_off


_default = None


def get() -> Oracle:
    """The oracle compiled without planted mistakes (built on first use)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default
