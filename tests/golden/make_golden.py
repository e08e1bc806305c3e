"""Write stored oracle results used by the GPU parity tests.

Every value written here comes from ``oracle`` (the CPU reference) applied to
instances from ``paper_1904_03621_gb300.instances``; nothing comes from the
CUDA library.  Usage (from the repository root):

    python tests/golden/make_golden.py plain_n20        # full 2^20 enumeration, S=10
    python tests/golden/make_golden.py int_n32          # full 2^32 enumeration, S=100
    python tests/golden/make_golden.py float_n48_sub    # 64 fixed-prefix subspaces of 2^24, S=1000
    python tests/golden/make_golden.py batched_sample   # 96 sampled instances of the 4096 batch, S=10
    python tests/golden/make_golden.py grad_sample      # 8 sampled n=28 instances, S=32, + gradients

Output files are gzip-compressed text, one record per line:
    <block> <rank> <energy> <state>
with energies written by repr() (exact round trip).
"""
from __future__ import annotations

import gzip
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1904_03621_gb300 import instances  # noqa: E402

# fixed-prefix subspaces of the n=48 instance: 24 fixed top bits, values drawn with seed 1
N48_FIXED_BITS = 24
N48_SUBSPACES = 64
N48_S = 1000

# sampled instances of the 4096-instance batch (indices drawn with seed 2)
BATCH_SAMPLE = 96
GRAD_SAMPLE = 8


def n48_prefixes():
    rng = np.random.default_rng(1)
    return sorted(int(v) for v in rng.choice(1 << N48_FIXED_BITS, size=N48_SUBSPACES, replace=False))


def batch_sample_indices():
    rng = np.random.default_rng(2)
    return sorted(int(v) for v in rng.choice(4096, size=BATCH_SAMPLE, replace=False))


def grad_sample_indices():
    rng = np.random.default_rng(2)
    return sorted(int(v) for v in rng.choice(256, size=GRAD_SAMPLE, replace=False))


def _write(path, header, blocks):
    with gzip.open(path, "wt") as f:
        for line in header:
            f.write("# " + line + "\n")
        for b, (en, st) in blocks:
            for k, (e, s) in enumerate(zip(en, st)):
                f.write(f"{b} {k} {repr(e.item())} {int(s)}\n")


def read(path):
    """{block: (energies, states)} from a golden file."""
    out = {}
    with gzip.open(path, "rt") as f:
        for line in f:
            if line.startswith("#"):
                continue
            b, k, e, s = line.split()
            out.setdefault(int(b), ([], []))
            out[int(b)][0].append(float(e) if ("." in e or "e" in e or "inf" in e) else int(e))
            out[int(b)][1].append(int(s))
    return {b: (np.array(v[0]), np.array(v[1], dtype=np.uint64)) for b, v in out.items()}


def make_plain_n20():
    o = oracle.get()
    J, h = instances.plain_n20()
    t = time.time()
    en, st = o.low_spectrum(J, h, 10)
    dt = time.time() - t
    _write(os.path.join(HERE, "plain_n20_S10.txt.gz"),
           ["instance plain_n20 seed 0 (n=20, J_ij~N(0,1), h_i~N(0,1), FP64), S=10, full enumeration",
            f"oracle {dt:.1f} s on {o.num_threads} threads"], [(0, (en, st))])


def make_int_n32():
    o = oracle.get()
    J, h = instances.int_n32()
    t = time.time()
    en, st = o.low_spectrum(J, h, 100)
    dt = time.time() - t
    _write(os.path.join(HERE, "int_n32_S100.txt.gz"),
           [f"instance int_n32 seed 0 (n=32, J uniform in {{-1,+1}}, h=0), S=100, full enumeration",
            f"oracle {dt:.0f} s on {o.num_threads} threads"], [(0, (en, st))])


def make_float_n48_sub():
    o = oracle.get()
    J, h = instances.float_n48()
    blocks = []
    t = time.time()
    for v in n48_prefixes():
        blocks.append((v, o.low_spectrum(J, h, N48_S, fixed_bits=N48_FIXED_BITS, fixed_value=v)))
    dt = time.time() - t
    _write(os.path.join(HERE, "float_n48_sub24_S1000.txt.gz"),
           [f"instance float_n48 seed 0; {N48_SUBSPACES} subspaces with the top {N48_FIXED_BITS} bits fixed "
            f"(values drawn with numpy default_rng(1)); block id = fixed value; S={N48_S}",
            f"oracle {dt:.0f} s on {o.num_threads} threads"], blocks)


def make_batched_sample():
    o = oracle.get()
    inst = instances.batched_4096()
    blocks = []
    t = time.time()
    for i in batch_sample_indices():
        J, h, _ = inst[i]
        blocks.append((i, o.low_spectrum(J, h, 10)))
    dt = time.time() - t
    _write(os.path.join(HERE, "batched_sample_S10.txt.gz"),
           [f"instances batched_4096 seed 0; {BATCH_SAMPLE} indices drawn with default_rng(2); block id = index; S=10",
            f"oracle {dt:.0f} s on {o.num_threads} threads"], blocks)


def make_grad_sample():
    o = oracle.get()
    inst, w = instances.grad_256()
    blocks = []
    t = time.time()
    for i in grad_sample_indices():
        J, h = inst[i]
        blocks.append((i, o.low_spectrum(J.astype(np.float64), h.astype(np.float64), 32)))
    dt = time.time() - t
    _write(os.path.join(HERE, "grad_sample_S32.txt.gz"),
           [f"instances grad_256 seed 0 (FP32 values widened to FP64); {GRAD_SAMPLE} indices drawn with "
            f"default_rng(2); block id = index; S=32",
            f"oracle {dt:.0f} s on {o.num_threads} threads"], blocks)


if __name__ == "__main__":
    jobs = {"plain_n20": make_plain_n20, "int_n32": make_int_n32, "float_n48_sub": make_float_n48_sub,
            "batched_sample": make_batched_sample, "grad_sample": make_grad_sample}
    for name in sys.argv[1:]:
        jobs[name]()
        print("wrote", name, flush=True)
