"""GPU direct sum (lens_direct_deflect) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens, synth
from helpers import alpha_rel_err

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec,tol", [(lens.FP64, 1e-10), (lens.FP32_BULK, 2e-5)])
def test_direct_matches_oracle(prec, tol):
    f = synth.c1_plain(seed=0)
    x = synth.random_rays(1, 3001, (-10, -10), (10, 10))  # ragged: not a multiple of a tile
    y, jac = lens.direct_deflect(T(f.stars), T(f.masses), 0.1, 0.25, T(x), prec=prec, jacobian=True)
    y_ref, jac_ref = oracle.deflect(f.stars, f.masses, 0.1, 0.25, x, jacobian=True)
    err = alpha_rel_err(y.cpu().numpy(), y_ref, x, 0.1, 0.25)
    assert err.max() < tol, err.max()
    dj = np.abs(jac.cpu().numpy() - jac_ref).max() / np.abs(jac_ref).max()
    assert dj < (1e-10 if prec == lens.FP64 else 1e-4), dj


def test_direct_far_from_origin_fp32():
    # float32 form keeps accuracy at |x| ~ 1e3 (split hi/lo coordinates)
    f = synth.config_uniform(seed=2, n=2000, kappa_star=0.45, kappa_s=0.0, gamma=0.45,
                             radius=1200.0)
    x = synth.random_rays(3, 2000, (900, -50), (1000, 50))
    y = lens.direct_deflect(T(f.stars), T(f.masses), 0.0, 0.45, T(x), prec=lens.FP32_BULK)
    y_ref = oracle.deflect(f.stars, f.masses, 0.0, 0.45, x)
    assert alpha_rel_err(y.cpu().numpy(), y_ref, x, 0.0, 0.45).max() < 2e-5


def test_direct_edge_cases():
    stars = np.array([[0.0, 0.0], [1.0, 0.0]])
    x = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 0.5]])
    for prec in (lens.FP64, lens.FP32_BULK):
        y = lens.direct_deflect(T(stars), T([1.0, 1.0]), 0.0, 0.0, T(x), prec=prec).cpu().numpy()
        y_ref = oracle.deflect(stars, [1.0, 1.0], 0.0, 0.0, x)
        np.testing.assert_allclose(y, y_ref, rtol=1e-6, atol=1e-7)
    # zero rays
    y = lens.direct_deflect(T(stars), T([1.0, 1.0]), 0.0, 0.0, T(np.zeros((0, 2))))
    assert y.shape == (0, 2)
