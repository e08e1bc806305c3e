"""Fitting couplings so that an instance's low spectrum matches a target (the differentiable
form used as intended): L-BFGS through LowSpectrumFn (forward search + backward kernel) on
n = 16..18 instances; the loss must not increase, must reach the tolerance, and the fitted
instance's spectrum computed by the oracle must equal the target."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from parity import assert_float_parity, tolerance
from paper_1904_03621_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fit():
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import fit as f
    return f


def perturbed(a, rng, scale):
    noise = np.triu(rng.standard_normal(a.shape), 1) if a.ndim == 2 else rng.standard_normal(a.shape)
    return a + scale * noise


@pytest.mark.parametrize("n,S,seed,scale,factor", [(16, 8, 0, 0.05, 1.0), (18, 16, 1, 0.1, 1.0),
                                                   (16, 4, 2, 0.0, 1.1)])
def test_fit_spectrum_to_target(fit, n, S, seed, scale, factor):
    import torch
    o = oracle.get()
    Jt, ht = instances.dense_gaussian(n, 3000 + seed)
    target = factor * o.low_spectrum(Jt, ht, S)[0]          # attainable: the spectrum of factor * (J, h)
    rng = np.random.default_rng(seed)
    J0, h0 = perturbed(np.triu(Jt, 1), rng, scale), perturbed(ht, rng, scale)
    J, h, losses = fit.fit_spectrum(torch.tensor(J0, device="cuda"), torch.tensor(h0, device="cuda"),
                                    torch.tensor(target, device="cuda"), steps=400, tol=1e-22)
    assert losses[0] > 1e-6
    assert all(b <= a * (1 + 1e-9) + 1e-24 for a, b in zip(losses, losses[1:])), losses
    assert losses[-1] < 1e-16, losses
    Jf, hf = J.cpu().numpy(), h.cpu().numpy()
    assert np.all(np.tril(Jf) == 0.0)
    en_o, st_o = o.low_spectrum(Jf, hf, S + 1)
    assert np.abs(en_o[:S] - target).max() <= tolerance(Jf, hf)
    # and the library agrees with the oracle on the fitted instance
    from paper_1904_03621_gb300 import api
    en, st = api.low_spectrum(J, h, S)
    assert_float_parity(o, Jf, hf, en.cpu().numpy(), api.states_u64(st), en_o, st_o)
