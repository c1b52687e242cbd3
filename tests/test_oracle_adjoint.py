"""Pins of the oracle's adjoint (gradient through Eq. 1) and light curve.

The oracle's gradient is written from the real-variable derivatives of Eq. 1;
it is pinned by central finite differences of the oracle's own forward map
(a different computation), and by the complex-variable identities
dL/dm_j = Re F(z_j), dL/dx_j = Re(m_j G_j), dL/dy_j = -Im(m_j G_j) with
F(w) = sum_r c_r/(z_r - w), G = F'(w), c = -(g1 + i g2) -- a separate
derivation written out here in numpy.
"""
import numpy as np
import pytest

import oracle
from paper_2211_00354_gb300 import synth


def small_field(seed=0, n=60):
    f = synth.config_uniform(seed=seed, n=n, kappa_star=0.3, kappa_s=0.2, gamma=0.4,
                             mass_range=(0.5, 1.5))
    rays = np.random.default_rng(seed + 1).uniform(-4, 4, (200, 2))
    return f, rays


def linear_loss(f, stars, masses, ks, g, rays, W):
    y = oracle.deflect(stars, masses, ks, g, rays)
    return float(np.sum(W * y))


def test_adjoint_matches_finite_differences():
    f, rays = small_field()
    W = np.random.default_rng(9).normal(size=rays.shape)
    gxy, gm, gkg = oracle.adjoint(f.stars, f.masses, rays, W)
    h = 1e-6
    rng = np.random.default_rng(3)
    for j in rng.choice(f.n, 12, replace=False):
        for k in range(2):
            sp = f.stars.copy(); sp[j, k] += h
            sm = f.stars.copy(); sm[j, k] -= h
            fd = (linear_loss(f, sp, f.masses, f.kappa_s, f.gamma, rays, W)
                  - linear_loss(f, sm, f.masses, f.kappa_s, f.gamma, rays, W)) / (2 * h)
            assert gxy[j, k] == pytest.approx(fd, rel=1e-6, abs=1e-7)
        mp = f.masses.copy(); mp[j] += h
        mm = f.masses.copy(); mm[j] -= h
        fd = (linear_loss(f, f.stars, mp, f.kappa_s, f.gamma, rays, W)
              - linear_loss(f, f.stars, mm, f.kappa_s, f.gamma, rays, W)) / (2 * h)
        assert gm[j] == pytest.approx(fd, rel=1e-6, abs=1e-7)
    for idx, (dk, dg) in enumerate([(h, 0), (0, h)]):
        fd = (linear_loss(f, f.stars, f.masses, f.kappa_s + dk, f.gamma + dg, rays, W)
              - linear_loss(f, f.stars, f.masses, f.kappa_s - dk, f.gamma - dg, rays, W)) / (2 * h)
        assert gkg[idx] == pytest.approx(fd, rel=1e-7)


def test_adjoint_matches_complex_form():
    f, rays = small_field(seed=4, n=80)
    g = np.random.default_rng(2).normal(size=rays.shape)
    gxy, gm, _ = oracle.adjoint(f.stars, f.masses, rays, g)
    c = -(g[:, 0] + 1j * g[:, 1])
    zr = rays[:, 0] + 1j * rays[:, 1]
    zs = f.stars[:, 0] + 1j * f.stars[:, 1]
    D = zr[None, :] - zs[:, None]
    F = np.sum(c[None, :] / D, axis=1)
    G = np.sum(c[None, :] / D ** 2, axis=1)
    np.testing.assert_allclose(gm, F.real, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(gxy[:, 0], (f.masses * G).real, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(gxy[:, 1], -(f.masses * G).imag, rtol=1e-11, atol=1e-12)


def test_light_curve_of_unlensed_gaussian_is_one():
    # y = x on a fine grid: a unit-normalised Gaussian source has mu = 1
    grid = synth.Grid(x0=-1.0, y0=-1.0, h=0.01, nx=200, ny=200)
    y = grid.corners().reshape(-1, 2)
    s = synth.light_curve_track(64, length=0.6)
    F = oracle.light_curve(y, grid.h ** 2, s, 0.05, trunc=6.0)
    np.testing.assert_allclose(F, 1.0, rtol=1e-6)


def test_light_curve_gradient_matches_finite_differences():
    rng = np.random.default_rng(8)
    y = rng.uniform(-0.5, 0.5, (400, 2))
    s = synth.light_curve_track(40, length=0.8)
    T = rng.uniform(0, 2, 40)
    w, sig = 1e-3, 0.05
    L0, F = oracle.light_curve_loss(y, w, s, sig, T, trunc=6.0)
    gy = oracle.light_curve_grad(y, w, s, sig, F, T, trunc=6.0)
    h = 1e-6
    for r in rng.choice(400, 10, replace=False):
        for k in range(2):
            yp = y.copy(); yp[r, k] += h
            ym = y.copy(); ym[r, k] -= h
            fd = (oracle.light_curve_loss(yp, w, s, sig, T)[0] - oracle.light_curve_loss(ym, w, s, sig, T)[0]) / (2 * h)
            # FD rounding noise ~ eps * L / h ~ 1e-8
            assert gy[r, k] == pytest.approx(fd, rel=1e-5, abs=5e-8)
