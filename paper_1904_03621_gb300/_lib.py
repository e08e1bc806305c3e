"""ctypes declarations of the C ABI in include/bf.h (argument marshalling only).

Loading fails loudly when libbf.so has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbf.so")

BF_OK, BF_EINVAL, BF_ECUDA, BF_EOVERFLOW, BF_ETIMEOUT, BF_EUNSUPPORTED, BF_EWORKSPACE = range(7)
BF_I32, BF_F32, BF_F64 = 0, 1, 2
BF_VARIANT_AUTO, BF_VARIANT_GRAY, BF_VARIANT_TC = 0, 1, 2

# every symbol include/bf.h declares
EXPORTS = ["bf_workspace_size", "bf_low_spectrum", "bf_autotune", "bf_low_spectrum_noalloc", "bf_batched_workspace_size",
           "bf_low_spectrum_batched", "bf_autotune_batched", "bf_low_spectrum_backward", "bf_qubo_workspace_size",
           "bf_low_spectrum_qubo", "bf_potts_workspace_size", "bf_low_spectrum_potts", "bf_instance_digest", "bf_cursor_bytes", "bf_cursor_init",
           "bf_cursor_workspace_size", "bf_cursor_step", "bf_cursor_state", "bf_workspace_status",
           "bf_last_profile", "bf_launch_count", "bf_issue_rates_workspace_size", "bf_measure_issue_rates",
           "bf_merge_lists", "bf_status_string", "bf_last_error_detail",
           "bf_version"]


class Options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("fixed_bits", ctypes.c_int32), ("fixed_value", ctypes.c_uint64),
                ("task_log2", ctypes.c_int32), ("grid_blocks", ctypes.c_int32), ("spill_log2", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("stall_test", ctypes.c_int32), ("inner_bits", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class TuneRecord(ctypes.Structure):
    _fields_ = [("opt", Options), ("configs_per_s", ctypes.c_double)]


class IssueRates(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int32), ("sm_clock_mhz", ctypes.c_double), ("iadd3_lanes_per_clk", ctypes.c_double),
                ("lop3_lanes_per_clk", ctypes.c_double), ("vmnmx_lanes_per_clk", ctypes.c_double),
                ("ffma_lanes_per_clk", ctypes.c_double)]


class BFError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {detail}")
        self.status = status


STATUS_NAMES = {0: "BF_OK", 1: "BF_EINVAL", 2: "BF_ECUDA", 3: "BF_EOVERFLOW", 4: "BF_ETIMEOUT",
                5: "BF_EUNSUPPORTED", 6: "BF_EWORKSPACE"}

_lib = None


def load(path: str | None = None):
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} not found: build the CUDA library first (paper_1904_03621_gb300.build.build())")
    lib = ctypes.CDLL(p)
    vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    lib.bf_workspace_size.restype = sz
    lib.bf_workspace_size.argtypes = [i32, i32, i32, ctypes.POINTER(Options)]
    lib.bf_low_spectrum.restype = i32
    lib.bf_low_spectrum.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, sz, ctypes.POINTER(Options), vp]
    lib.bf_autotune.restype = i32
    lib.bf_autotune.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, sz, ctypes.POINTER(Options), vp,
                                ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(TuneRecord),
                                i32, ctypes.POINTER(ctypes.c_int)]
    lib.bf_low_spectrum_noalloc.restype = i32
    lib.bf_low_spectrum_noalloc.argtypes = [vp, vp, i32, i32, i32, vp, vp, ctypes.POINTER(Options), vp]
    lib.bf_batched_workspace_size.restype = sz
    lib.bf_batched_workspace_size.argtypes = [i32, i32, i32, i32, ctypes.POINTER(Options)]
    lib.bf_low_spectrum_batched.restype = i32
    lib.bf_low_spectrum_batched.argtypes = [i32, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, sz,
                                            ctypes.POINTER(Options), vp]
    lib.bf_autotune_batched.restype = i32
    lib.bf_autotune_batched.argtypes = [i32, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, sz, vp,
                                        ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_float)]
    lib.bf_low_spectrum_backward.restype = i32
    lib.bf_low_spectrum_backward.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, i32, vp]
    lib.bf_qubo_workspace_size.restype = sz
    lib.bf_qubo_workspace_size.argtypes = [i32, i32, i32, ctypes.POINTER(Options)]
    lib.bf_low_spectrum_qubo.restype = i32
    lib.bf_low_spectrum_qubo.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, sz, ctypes.POINTER(Options), vp]
    lib.bf_potts_workspace_size.restype = sz
    lib.bf_potts_workspace_size.argtypes = [i32, i32, i32, i32, ctypes.POINTER(Options)]
    lib.bf_low_spectrum_potts.restype = i32
    lib.bf_low_spectrum_potts.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp, vp, sz, ctypes.POINTER(Options), vp]
    lib.bf_instance_digest.restype = ctypes.c_uint64
    lib.bf_instance_digest.argtypes = [vp, vp, i32, i32]
    lib.bf_cursor_bytes.restype = sz
    lib.bf_cursor_bytes.argtypes = [i32]
    lib.bf_cursor_init.restype = i32
    lib.bf_cursor_init.argtypes = [vp, sz, i32, i32, i32, i32, ctypes.c_uint64]
    lib.bf_cursor_workspace_size.restype = sz
    lib.bf_cursor_workspace_size.argtypes = [vp, sz, ctypes.POINTER(Options)]
    lib.bf_cursor_step.restype = i32
    lib.bf_cursor_step.argtypes = [vp, sz, vp, vp, i32, vp, sz, ctypes.POINTER(Options), vp]
    lib.bf_cursor_state.restype = i32
    lib.bf_cursor_state.argtypes = [vp, sz, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), vp, vp,
                                    ctypes.POINTER(ctypes.c_int)]
    lib.bf_merge_lists.restype = i32
    lib.bf_merge_lists.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp), i32, i32, i32, vp, vp]
    lib.bf_workspace_status.restype = i32
    lib.bf_workspace_status.argtypes = [vp, vp]
    lib.bf_status_string.restype = ctypes.c_char_p
    lib.bf_status_string.argtypes = [i32]
    lib.bf_last_error_detail.restype = ctypes.c_char_p
    lib.bf_last_error_detail.argtypes = []
    lib.bf_version.restype = ctypes.c_char_p
    lib.bf_last_profile.restype = i32
    lib.bf_last_profile.argtypes = [ctypes.POINTER(ctypes.c_float)]
    lib.bf_launch_count.restype = ctypes.c_int64
    lib.bf_launch_count.argtypes = []
    lib.bf_issue_rates_workspace_size.restype = sz
    lib.bf_issue_rates_workspace_size.argtypes = []
    lib.bf_measure_issue_rates.restype = i32
    lib.bf_measure_issue_rates.argtypes = [vp, sz, ctypes.POINTER(IssueRates), vp]
    if path is None:
        _lib = lib
    return lib


def check(status: int, lib=None):
    if status != BF_OK:
        lib = lib or load()
        raise BFError(status, lib.bf_last_error_detail().decode())
