"""bf_low_spectrum_batched on the GPU against the oracle."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from parity import assert_float_parity, assert_int_equal
from paper_1904_03621_gb300 import instances

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def mixed_batch(count, seed, n_lo=10, n_hi=20):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        if i % 2 == 0:
            J, h = instances.dense_gaussian(n, 1000 + i, h_std=0.5)
        else:
            J, h = instances.chimera_pm1(n, rng)
            J, h = J.astype(np.float64), h.astype(np.float64)
        out.append((J, h))
    return out


def check_all(o, insts, en, st, S):
    for b, (J, h) in enumerate(insts):
        n = J.shape[0]
        if np.issubdtype(J.dtype, np.integer):
            en_o, st_o = o.low_spectrum(J, h, S)
            assert_int_equal(en[b], st[b], en_o, st_o)
        else:
            S1 = min(S + 1, 1 << n)
            en_o, st_o = o.low_spectrum(J, h, S1)
            assert_float_parity(o, J, h, en[b], st[b], en_o, st_o)


@pytest.mark.parametrize("S", [1, 10, 64])
def test_batched_mixed_float(bf, o, S):
    insts = mixed_batch(40, S)
    args = bf.pack_batch(insts)
    en, st = bf.low_spectrum_batched(*args[:5], S, n_max=args[5])
    check_all(o, insts, en.cpu().numpy(), bf.states_u64(st).reshape(en.shape), S)


@pytest.mark.parametrize("S", [5, 33])
def test_batched_scales_and_windows(bf, o, S):
    """One batch whose instances differ in scale by 18 orders of magnitude (the per-instance
    fixed-point exponent q from about -30 to +60), plus integer-valued float instances
    (residual 0, no window) and near-integer ones (tiny residuals, a window of a few units):
    the quantisation, the residual words and the final re-evaluation of every instance must
    reproduce the oracle.  n from 10 (the exact sample) to 22."""
    rng = np.random.default_rng(400 + S)
    insts = []
    for i, scale in enumerate([1e-9, 1e-3, 1.0, 1e3, 1e9] * 3):
        n = int(rng.integers(10, 23))
        J, h = instances.dense_gaussian(n, 500 + i, h_std=0.7)
        insts.append((J * scale, h * scale))
    for i in range(6):
        n = int(rng.integers(10, 23))
        J, h = instances.dense_pm1(n, 600 + i)
        J, h = J.astype(np.float64), h.astype(np.float64)
        if i % 2:   # near-integer couplings: residuals of about 1e-7
            N = np.triu(rng.normal(0.0, 1e-7, J.shape), 1)
            J = J + N + N.T
        insts.append((J, h))
    args = bf.pack_batch(insts)
    en, st = bf.low_spectrum_batched(*args[:5], S, n_max=args[5], task_log2=21)
    check_all(o, insts, en.cpu().numpy(), bf.states_u64(st).reshape(en.shape), S)


def test_batched_int(bf, o):
    rng = np.random.default_rng(7)
    insts = [instances.dense_pm1(int(rng.integers(10, 22)), 50 + i) for i in range(24)]
    import torch
    args = bf.pack_batch(insts, dtype=torch.int32)
    en, st = bf.low_spectrum_batched(*args[:5], 17, n_max=args[5])
    check_all(o, insts, en.cpu().numpy(), bf.states_u64(st).reshape(en.shape), 17)


def test_batched_float32_uniform_n(bf, o):
    import torch
    insts = [(J.astype(np.float32), h.astype(np.float32)) for J, h in
             (instances.dense_gaussian(22, 70 + i) for i in range(6))]
    args = bf.pack_batch(insts, dtype=torch.float32)
    en, st = bf.low_spectrum_batched(*args[:5], 32, n_max=args[5], task_log2=21)
    ref = [(J.astype(np.float64), h.astype(np.float64)) for J, h in insts]
    check_all(o, ref, en.cpu().numpy(), bf.states_u64(st).reshape(en.shape), 32)


def test_batched_graph_capture(bf, o):
    import torch
    insts = mixed_batch(16, 99, 12, 18)
    J, Jo, h, ho, n, n_max = bf.pack_batch(insts)
    S = 8
    ws = torch.empty(bf.batched_workspace_size(len(insts), n_max, S, torch.float64), dtype=torch.uint8,
                     device="cuda")
    en = torch.empty(len(insts), S, dtype=torch.float64, device="cuda")
    st = torch.empty(len(insts), S, dtype=torch.int64, device="cuda")
    bf.low_spectrum_batched(J, Jo, h, ho, n, S, n_max=n_max, workspace=ws, out=(en, st))   # warm-up
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bf.low_spectrum_batched(J, Jo, h, ho, n, S, n_max=n_max, workspace=ws, out=(en, st), check=False)
    for _ in range(2):
        en.zero_()
        st.zero_()
        g.replay()
        torch.cuda.synchronize()
        check_all(o, insts, en.cpu().numpy(), bf.states_u64(st).reshape(en.shape), S)


def test_batched_invalid_n(bf):
    import torch
    from paper_1904_03621_gb300 import _lib
    insts = mixed_batch(4, 3, 12, 14)
    J, Jo, h, ho, n, n_max = bf.pack_batch(insts)
    n_bad = n.clone()
    n_bad[2] = 40            # beyond n_max
    with pytest.raises(_lib.BFError) as e:
        bf.low_spectrum_batched(J, Jo, h, ho, n_bad, 4, n_max=n_max)
    assert e.value.status == _lib.BF_EINVAL
    with pytest.raises(_lib.BFError) as e:
        bf.low_spectrum_batched(J, Jo, h, ho, n, 65, n_max=n_max)
    assert e.value.status == _lib.BF_EINVAL


def test_batched_4096_sample(bf):
    """The 4096-instance workload (2048 dense, 2048 Chimera, n in [16, 28], S = 10) in one
    call; 96 sampled instances against stored oracle results, all instances by properties."""
    import importlib.util
    path = os.path.join(GOLDEN, "batched_sample_S10.txt.gz")
    if not os.path.exists(path):
        pytest.skip("golden not generated")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    gold = mg.read(path)
    insts = instances.batched_4096()
    args = bf.pack_batch(insts)
    en, st = bf.low_spectrum_batched(*args[:5], 10, n_max=args[5])
    en = en.cpu().numpy()
    st = bf.states_u64(st).reshape(en.shape)
    o = oracle.get()
    for i, (en_o, st_o) in gold.items():
        J, h, kind = insts[i]
        if kind == "sparse":
            assert_int_equal(en[i], st[i], en_o, st_o)
        else:
            assert_float_parity(o, J, h, en[i], st[i], en_o, st_o)
    # every instance, by properties that hold at any size: returned energies are the oracle's
    # energies of the returned states, ascending by (E, c), no duplicates; and on 256 sampled
    # instances, every single-spin-flip neighbour below the S-th energy is returned
    from parity import tolerance
    rng = np.random.default_rng(11)
    closure = set(rng.choice(len(insts), 256, replace=False).tolist())
    for i, (J, h, kind) in enumerate(insts):
        n = J.shape[0]
        tol = 0.0 if kind == "sparse" else tolerance(J, h)
        e_i, s_i = en[i], st[i]
        assert len(set(s_i.tolist())) == len(s_i), i
        assert np.all(np.diff(e_i) >= 0), i
        for k in range(len(s_i)):
            assert abs(o.energy(J, h, int(s_i[k])) - e_i[k]) <= tol, (i, k)
        if i in closure:
            members = set(int(c) for c in s_i)
            for c in s_i:
                for b in range(n):
                    nb = int(c) ^ (1 << b)
                    if o.energy(J, h, nb) < e_i[-1] - tol:
                        assert nb in members, (i, int(c), b)


def test_batched_autotune(bf, o):
    """The autotuner returns one of its candidates, and later default calls (which use the
    cached choice) give the same exact results as explicit options."""
    insts = mixed_batch(24, 123, 16, 24)
    args = bf.pack_batch(insts)
    tuned = bf.autotune_batched(*args[:5], 10, n_max=args[5])
    assert tuned["task_log2"] in (21, 23, 25, 27) and tuned["grid_blocks"] > 0 and tuned["ms"] > 0
    en_d, st_d = bf.low_spectrum_batched(*args[:5], 10, n_max=args[5])
    en_e, st_e = bf.low_spectrum_batched(*args[:5], 10, n_max=args[5], task_log2=25, grid_blocks=152)
    assert np.array_equal(bf.states_u64(st_d), bf.states_u64(st_e))
    check_all(o, insts, en_d.cpu().numpy(), bf.states_u64(st_d).reshape(en_d.shape), 10)
