"""Pins of the oracle's lensing potential (Sec. 2.5): its gradient is x - y
of the (independently pinned) direct-sum lens equation, a ring of masses
gives M ln R at its centre, a single mass m ln|x - x0|, and the smooth
field alone kappa_s |x|^2 / 2 + gamma (x1^2 - x2^2) / 2."""
import numpy as np
import pytest

import oracle
from paper_2211_00354_gb300 import synth


def test_gradient_is_x_minus_y():
    f = synth.config_uniform(seed=2, n=200, kappa_star=0.4, kappa_s=0.15, gamma=0.25)
    rng = np.random.default_rng(3)
    x = rng.uniform(-3, 3, size=(40, 2))
    y = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    h = 1e-5
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        g = (oracle.potential(f.stars, f.masses, f.kappa_s, f.gamma, x + e) -
             oracle.potential(f.stars, f.masses, f.kappa_s, f.gamma, x - e)) / (2 * h)
        np.testing.assert_allclose(g, x[:, k] - y[:, k], rtol=1e-6, atol=1e-6)


def test_ring_and_single_mass():
    n, R, M = 64, 1.7, 3.0
    th = 2 * np.pi * np.arange(n) / n
    ring = np.stack([0.3 + R * np.cos(th), -0.2 + R * np.sin(th)], axis=1)
    psi = oracle.potential(ring, np.full(n, M / n), 0.0, 0.0, np.array([[0.3, -0.2]]))
    assert psi[0] == pytest.approx(M * np.log(R), rel=1e-13)
    x = np.array([[1.0, 2.0], [-0.5, 0.25], [0.7, -0.4]])
    psi = oracle.potential(np.array([[0.7, -0.4]]), np.array([2.5]), 0.0, 0.0, x)
    assert psi[0] == pytest.approx(2.5 * np.log(np.hypot(0.3, 2.4)), rel=1e-14)
    assert psi[1] == pytest.approx(2.5 * np.log(np.hypot(1.2, 0.65)), rel=1e-14)
    assert psi[2] == 0.0  # the star itself contributes nothing


def test_smooth_field_alone():
    x = np.array([[1.5, -0.5], [0.0, 2.0]])
    psi = oracle.potential(np.zeros((1, 2)) + 100.0, np.zeros(1), 0.2, 0.3, x)
    ref = 0.5 * 0.2 * (x[:, 0] ** 2 + x[:, 1] ** 2) + 0.5 * 0.3 * (x[:, 0] ** 2 - x[:, 1] ** 2)
    np.testing.assert_allclose(psi, ref, rtol=1e-15)
