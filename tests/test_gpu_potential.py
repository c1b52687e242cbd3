"""Lensing potential through the plan's expansions (lens_potential) against
the oracle's direct sum: uniform and clustered fields (V, X, U and W lists
all in use), float64 and float32-bulk plans, and its gradient against the
plan's own deflections.  The tolerance is relative to the scale
S = sum_i m_i (1 + |ln|x - x_i||) of the terms summed at each ray."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens, synth

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def term_scale(stars, masses, x):
    d = np.hypot(x[:, None, 0] - stars[None, :, 0], x[:, None, 1] - stars[None, :, 1])
    with np.errstate(divide="ignore"):
        return np.sum(masses[None, :] * (1.0 + np.abs(np.log(np.where(d > 0, d, 1.0)))), axis=1)


def clustered(seed, n_clusters=40, per=200, a=0.05, R=6.0):
    rng = np.random.default_rng(seed)
    cen = rng.uniform(-R, R, size=(n_clusters, 2))
    u = rng.uniform(0.0, 0.95, size=(n_clusters, per))
    r = a * np.sqrt(u / (1.0 - u))
    th = rng.uniform(0, 2 * np.pi, size=(n_clusters, per))
    st = cen[:, None, :] + np.stack([r * np.cos(th), r * np.sin(th)], axis=-1)
    st = st.reshape(-1, 2)
    return st, rng.lognormal(0.0, 0.5, size=st.shape[0])


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
@pytest.mark.parametrize("prec,p,tol", [(lens.FP64, 40, 1e-12), (lens.FP32_BULK, 16, 1e-7)])
def test_potential_against_direct_sum(kind, prec, p, tol):
    if kind == "uniform":
        f = synth.config_uniform(seed=7, n=3000, kappa_star=0.4, kappa_s=0.1, gamma=0.3)
        stars, masses, ks, g = f.stars, f.masses, f.kappa_s, f.gamma
        box = (-4.0, 4.0, -4.0, 4.0)
    else:
        stars, masses = clustered(8)
        ks, g = 0.0, 0.2
        box = (-5.0, 5.0, -5.0, 5.0)
    rng = np.random.default_rng(9)
    x = np.stack([rng.uniform(box[0], box[1], 3000), rng.uniform(box[2], box[3], 3000)], axis=1)
    # rays on top of cluster members too
    x[:50] = stars[rng.choice(stars.shape[0], 50, replace=False)] + 1e-6
    x = x[(x[:, 0] > box[0]) & (x[:, 0] < box[1]) & (x[:, 1] > box[2]) & (x[:, 1] < box[3])]
    with lens.LensFMM(T(stars), T(masses), ks, g, p=p, leaf_size=16, prec=prec,
                      target_box=box) as P:
        psi = P.potential(T(x)).cpu().numpy()
        info = P.info()
    ref = oracle.potential(stars, masses, ks, g, x)
    err = np.abs(psi - ref) / term_scale(stars, masses, x)
    print("%s %s: levels %d, V %d, X %d, W %d, max rel err %.2e"
          % (kind, "fp64" if prec == lens.FP64 else "fp32-bulk", info["levels"], info["n_v"],
             info["n_x"], info["n_w"], err.max()))
    if kind == "clustered":
        assert info["n_x"] > 0 and info["n_w"] > 0
    assert err.max() < tol


def test_potential_gradient_matches_deflection():
    f = synth.config_uniform(seed=10, n=2000, kappa_star=0.3, kappa_s=0.2, gamma=0.1)
    box = (-3.0, 3.0, -3.0, 3.0)
    rng = np.random.default_rng(11)
    x = rng.uniform(-2.5, 2.5, size=(500, 2))
    h = 1e-5
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=40, leaf_size=8,
                      prec=lens.FP64, target_box=box) as P:
        y = P.deflect(T(x)).cpu().numpy()
        for k in range(2):
            e = np.zeros(2)
            e[k] = h
            gk = (P.potential(T(x + e)).cpu().numpy() - P.potential(T(x - e)).cpu().numpy()) / (2 * h)
            np.testing.assert_allclose(gk, x[:, k] - y[:, k], rtol=1e-5, atol=1e-5)


def test_potential_outside_target_fails():
    f = synth.config_uniform(seed=12, n=100, kappa_star=0.3, kappa_s=0.0, gamma=0.0)
    with lens.LensFMM(T(f.stars), T(f.masses), 0.0, 0.0, p=16, leaf_size=8, prec=lens.FP64,
                      target_box=(-1.0, 1.0, -1.0, 1.0)) as P:
        with pytest.raises(lens.LensError) as ei:
            P.potential(T(np.array([[1e6, 0.0]])))
        assert ei.value.status == lens.LENS_EDOMAIN
