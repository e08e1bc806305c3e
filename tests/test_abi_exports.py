"""The C ABI library loads without a GPU and exports every function include/*.h declares."""
from __future__ import annotations

import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)          # drop comments
        for m in re.finditer(r"\b(bf_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_function():
    from paper_1904_03621_gb300 import build, _lib
    build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    declared = declared_functions()
    assert len(declared) >= 10
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert set(_lib.EXPORTS) == declared, "ctypes declarations and the header differ"


def test_host_only_calls_without_gpu():
    from paper_1904_03621_gb300 import _lib
    lib = _lib.load()
    assert lib.bf_version().startswith(b"libbf")
    assert lib.bf_status_string(_lib.BF_EOVERFLOW) == b"BF_EOVERFLOW"
    # argument validation happens on the host before any device work
    st = lib.bf_low_spectrum(None, None, 0, 1, _lib.BF_F64, None, None, None, 0, None, None)
    assert st == _lib.BF_EINVAL
    st = lib.bf_low_spectrum_backward(None, None, None, 0, 1, None, None, None, None, _lib.BF_F64, None)
    assert st == _lib.BF_EINVAL
    assert lib.bf_last_error_detail() != b""
    assert lib.bf_launch_count() >= 0


def test_graph_to_dense_marshalling():
    """Dict graph -> dense (J, h): fields from (i, i), pairs accumulated into the upper
    triangle in sorted-label order, dtype int32 for integer weights."""
    import numpy as np
    from paper_1904_03621_gb300.graph import graph_to_dense
    J, h, nodes = graph_to_dense({("b", "a"): 2, ("a", "b"): 3, ("c", "c"): -1, ("a", "a"): 4})
    assert nodes == ["a", "b", "c"]
    assert J.dtype == np.int32 and h.dtype == np.int32
    assert J.tolist() == [[0, 5, 0], [0, 0, 0], [0, 0, 0]]
    assert h.tolist() == [4, 0, -1]
    J, h, _ = graph_to_dense({(1, 2): 0.5})
    assert J.dtype == np.float64 and J[0, 1] == 0.5
