"""Backward kernel and autograd functions on the GPU against the oracle's gradient and
central finite differences of the GPU forward."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
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


def test_backward_kernel_vs_oracle(bf, o):
    import torch
    rng = np.random.default_rng(5)
    n_list = [1, 5, 17, 28, 64]
    S = 37
    states = np.stack([rng.integers(0, 1 << min(n, 63), S, dtype=np.uint64) for n in n_list])
    if 64 in n_list:
        states[-1] |= np.uint64(1) << np.uint64(63)
    g = rng.uniform(-1, 1, (len(n_list), S))
    dJ_o, dh_o, J_off, h_off = o.grad(n_list, states, g)
    dev = "cuda"
    for dt in (torch.float64, torch.float32):
        dJ, dh = bf.low_spectrum_backward(torch.from_numpy(states.view(np.int64)).to(dev),
                                          torch.from_numpy(g).to(dev),
                                          torch.tensor(n_list, dtype=torch.int32, device=dev),
                                          torch.from_numpy(J_off).to(dev), torch.from_numpy(h_off).to(dev),
                                          dJ_o.size, dh_o.size, dtype=dt)
        tol = 1e-12 * S if dt == torch.float64 else 1e-5 * S
        assert np.abs(dJ.cpu().numpy() - dJ_o).max() <= tol
        assert np.abs(dh.cpu().numpy() - dh_o).max() <= tol


def test_autograd_single(bf, o):
    import torch
    J, h = instances.dense_gaussian(20, 11)
    S = 16
    w = np.random.default_rng(3).uniform(0, 1, S)
    Jt = torch.tensor(J, device="cuda", requires_grad=True)
    ht = torch.tensor(h, device="cuda", requires_grad=True)
    en, st = bf.LowSpectrumFn.apply(Jt, ht, S)
    loss = (torch.tensor(w, device="cuda") * en).sum()
    loss.backward()
    states = bf.states_u64(st)
    dJ_o, dh_o, _, _ = o.grad([20], states.reshape(1, -1), w.reshape(1, -1))
    assert np.abs(Jt.grad.cpu().numpy().ravel() - dJ_o).max() < 1e-11
    assert np.abs(ht.grad.cpu().numpy() - dh_o).max() < 1e-11
    # central finite differences of the loss on a few couplings (the ground states do not change)
    en_all, _ = o.low_spectrum(J, h, S + 1)
    gaps = np.diff(en_all)
    assert gaps.min() > 4e-4, "instance chosen with non-degenerate low levels"
    step = 1e-4
    for (i, j) in [(0, 1), (3, 17), (18, 19)]:
        vals = []
        for sgn in (1, -1):
            Jp = J.copy()
            Jp[i, j] += sgn * step
            e, _ = bf.low_spectrum(torch.tensor(Jp, device="cuda"), torch.tensor(h, device="cuda"), S)
            vals.append(float((w * e.cpu().numpy()).sum()))
        fd = (vals[0] - vals[1]) / (2 * step)
        assert abs(fd - Jt.grad[i, j].item()) < 1e-6


def test_grad_256_workload(bf, o):
    """256 fully connected n=28 instances (FP32 J, h), S=32, L = sum_k w_k E_k: batched forward
    against stored oracle results, backward against the oracle gradient at the returned states,
    and central finite differences (step 1e-4) on 16 parameters of every instance."""
    import importlib.util
    import torch
    inst, w = instances.grad_256()
    S = 32
    Jp, Jo, hp, ho, n, n_max = bf.pack_batch(inst, dtype=torch.float32)
    Jp.requires_grad_(True)
    hp.requires_grad_(True)
    en, st = bf.LowSpectrumBatchedFn.apply(Jp, hp, Jo, ho, n, S, n_max)
    wt = torch.tensor(w, device="cuda")
    (wt * en).sum().backward()
    states = bf.states_u64(st).reshape(en.shape)
    en_np = en.detach().cpu().numpy()
    # forward vs stored oracle results
    path = os.path.join(GOLDEN, "grad_sample_S32.txt.gz")
    if os.path.exists(path):
        spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
        mg = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mg)
        from parity import assert_float_parity
        for i, (en_o, st_o) in mg.read(path).items():
            J, h = inst[i]
            assert_float_parity(o, J.astype(np.float64), h.astype(np.float64), en_np[i], states[i], en_o, st_o)
    # backward vs oracle gradient at the returned states
    dJ_o, dh_o, _, _ = o.grad([28] * len(inst), states, w)
    assert np.abs(Jp.grad.cpu().numpy().astype(np.float64) - dJ_o).max() < 1e-4
    assert np.abs(hp.grad.cpu().numpy().astype(np.float64) - dh_o).max() < 1e-4
    # central finite differences in FP64 on 16 parameters (all instances at once)
    J64 = [(J.astype(np.float64), h.astype(np.float64)) for J, h in inst]
    base = bf.pack_batch(J64, dtype=torch.float64)
    en1, _ = bf.low_spectrum_batched(*base[:5], S + 1, n_max=base[5])
    gaps = np.diff(en1.cpu().numpy(), axis=1)
    ok = gaps.min(axis=1) >= 4e-4
    rng = np.random.default_rng(2)
    pairs = set()
    while len(pairs) < 16:
        i, j = sorted(rng.choice(28, 2, replace=False))
        pairs.add((int(i), int(j)))
    step = 1e-4
    checked = 0
    gJ = Jp.grad.cpu().numpy().astype(np.float64).reshape(len(inst), 28, 28)
    for (i, j) in sorted(pairs):
        L = []
        for sgn in (1, -1):
            Jpert = base[0].clone()
            offs = torch.arange(len(inst), device="cuda", dtype=torch.int64) * 28 * 28 + i * 28 + j
            Jpert[offs] += sgn * step
            e, _ = bf.low_spectrum_batched(Jpert, *base[1:5], S, n_max=base[5])
            L.append((w * e.cpu().numpy()).sum(axis=1))
        fd = (L[0] - L[1]) / (2 * step)
        err = np.abs(fd - gJ[:, i, j])[ok]
        assert err.max() < 1e-6, f"pair {(i, j)}: max |FD - grad| = {err.max()}"
        checked += int(ok.sum())
    assert checked >= 16 * 200, f"only {checked} entries had non-degenerate levels"
