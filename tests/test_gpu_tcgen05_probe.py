"""The tcgen05 forms the tensor-core screen relies on, checked exactly on the GPU:
the BF16 MMA with the kernel's shared-memory descriptors, and the sm_103a reducing TMEM
load (its min / max equal the reductions of the loaded columns)."""
from __future__ import annotations

import os
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tcgen05_mma_and_reducing_load_exact():
    src = os.path.join(HERE, "cuda", "tcgen05_probe.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "tcgen05_probe")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", src, "-o", exe],
                       check=True, capture_output=True, text=True)
        res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "D mismatches=0" in res.stdout and "min mismatches=0" in res.stdout and "max mismatches=0" in res.stdout
