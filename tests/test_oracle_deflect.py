"""Pins of the oracle's Eq. 1 direct sum (lens equation with kappa_s, gamma).

Each test checks the oracle against something it does not compute itself:
closed forms of the Cauchy sum, finite differences, and algebraic
invariants.  A dropped term, swapped component, wrong sign of the smooth
field or of the shear, or a transposed Jacobian fails one of them.
"""
import numpy as np
import pytest

import oracle
from paper_2211_00354_gb300 import synth


def test_single_point_lens_closed_form():
    # Eq. 1 with one lens of mass m at x_1: alpha = m (x - x_1)/|x - x_1|^2
    rng = np.random.default_rng(1)
    x = rng.uniform(-3, 3, (200, 2))
    m, c = 0.7, np.array([0.3, -0.2])
    ks, g = 0.15, -0.25
    y, al = oracle.deflect(c[None], [m], ks, g, x, alpha=True)
    d = x - c
    expect = m * d / np.sum(d * d, axis=1)[:, None]
    np.testing.assert_allclose(al, expect, rtol=1e-14, atol=0)
    np.testing.assert_allclose(y[:, 0], (1 - ks - g) * x[:, 0] - expect[:, 0], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(y[:, 1], (1 - ks + g) * x[:, 1] - expect[:, 1], rtol=1e-13, atol=1e-14)


def ngon(N, R, phase=0.3):
    t = phase + 2 * np.pi * np.arange(N) / N
    return np.stack([R * np.cos(t), R * np.sin(t)], axis=1)


@pytest.mark.parametrize("N,R", [(3, 1.0), (12, 2.5), (64, 10.0)])
def test_regular_polygon_closed_form(N, R):
    # sum_k 1/(z - R w^k e^{i phase}) is the log-derivative of z^N - (R e^{i phase})^N,
    # so f(z) = N z^{N-1} / (z^N - c^N) with c = R e^{i phase}; alpha = conj(m f).
    m, phase = 1.3, 0.3
    stars = ngon(N, R, phase)
    rng = np.random.default_rng(N)
    x = np.concatenate([rng.uniform(-2 * R, 2 * R, (300, 2)), rng.uniform(-0.3 * R, 0.3 * R, (100, 2))])
    _, al, jac = oracle.deflect(stars, np.full(N, m), 0.0, 0.0, x, alpha=True, jacobian=True)
    z = x[:, 0] + 1j * x[:, 1]
    cN = (R * np.exp(1j * phase)) ** N
    f = m * N * z ** (N - 1) / (z ** N - cN)
    np.testing.assert_allclose(al[:, 0] + 1j * al[:, 1], np.conj(f), rtol=1e-11, atol=1e-13 * N * m / R)
    # Jacobian: dy/dx = diag(a, b) - [[Re f', -Im f'], [-Im f', -Re f']]
    fp = m * N * z ** (N - 2) * (-(z ** N) - (N - 1) * cN) / (z ** N - cN) ** 2
    scale = np.maximum(np.abs(fp), 1e-3)
    np.testing.assert_allclose(jac[:, 0, 0], 1 - fp.real, rtol=0, atol=1e-10 * scale.max())
    np.testing.assert_allclose(jac[:, 0, 1], fp.imag, rtol=0, atol=1e-10 * scale.max())
    np.testing.assert_allclose(jac[:, 1, 0], fp.imag, rtol=0, atol=1e-10 * scale.max())
    np.testing.assert_allclose(jac[:, 1, 1], 1 + fp.real, rtol=0, atol=1e-10 * scale.max())


def test_ring_has_no_interior_field():
    # 2D shell theorem (Sec. 2.3): a ring of many equal lenses deflects nothing deep inside
    N, R = 256, 50.0
    stars = ngon(N, R)
    x = np.random.default_rng(0).uniform(-10, 10, (100, 2))
    _, al = oracle.deflect(stars, np.ones(N), 0, 0, x, alpha=True)
    assert np.abs(al).max() < 1e-15 * N / R * 1e3  # (|z|/R)^(N-1) ~ 1e-180


def test_jacobian_matches_finite_differences():
    f = synth.config_uniform(seed=5, n=300, kappa_star=0.3, kappa_s=0.2, gamma=0.35)
    x = np.random.default_rng(7).uniform(-5, 5, (60, 2))
    _, jac = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x, jacobian=True)
    h = 1e-6
    for k in range(2):
        e = np.zeros(2); e[k] = h
        yp = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x + e)
        ym = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x - e)
        fd = (yp - ym) / (2 * h)
        np.testing.assert_allclose(jac[:, :, k], fd, rtol=1e-5, atol=1e-6)


def test_superposition_and_mass_scaling():
    rng = np.random.default_rng(11)
    A = rng.uniform(-5, 5, (40, 2)); B = rng.uniform(-5, 5, (70, 2))
    mA, mB = rng.uniform(0.1, 1, 40), rng.uniform(0.1, 1, 70)
    x = rng.uniform(-6, 6, (50, 2))
    _, aA = oracle.deflect(A, mA, 0, 0, x, alpha=True)
    _, aB = oracle.deflect(B, mB, 0, 0, x, alpha=True)
    _, aAB = oracle.deflect(np.concatenate([A, B]), np.concatenate([mA, mB]), 0, 0, x, alpha=True)
    np.testing.assert_allclose(aAB, aA + aB, rtol=1e-12, atol=1e-12)
    _, a2 = oracle.deflect(A, 2.5 * mA, 0, 0, x, alpha=True)
    np.testing.assert_allclose(a2, 2.5 * aA, rtol=1e-13, atol=0)
    # translation invariance of alpha
    t = np.array([3.0, -1.5])
    _, aT = oracle.deflect(A + t, mA, 0, 0, x + t, alpha=True)
    np.testing.assert_allclose(aT, aA, rtol=1e-10, atol=1e-12)


def test_self_interaction_skipped():
    stars = np.array([[0.0, 0.0], [1.0, 0.0]])
    _, al = oracle.deflect(stars, [1.0, 1.0], 0, 0, stars, alpha=True)
    np.testing.assert_allclose(al, [[-1.0, 0.0], [1.0, 0.0]], rtol=1e-15)


def test_uniform_disk_mean_field_is_kappa_x():
    # Expected deflection inside a uniform disk of lenses is kappa_* x (shell
    # theorem); statistical, checked through the median slope on a fixed seed.
    f = synth.config_uniform(seed=2, n=20000, kappa_star=0.4, kappa_s=0, gamma=0)
    x = np.random.default_rng(3).uniform(-20, 20, (3000, 2))
    _, al = oracle.deflect(f.stars, f.masses, 0, 0, x, alpha=True)
    slope = np.median(np.sum(al * x, axis=1) / np.sum(x * x, axis=1))
    assert abs(slope - 0.4) < 0.04
