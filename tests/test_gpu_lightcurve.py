"""The Gaussian-source light curve on the GPU (lens_light_curve,
lens_light_curve_grad), whose Gaussians are float-float on the float32 pipe
(the exponential by Tang's table-driven method): single-term cases against
float64 exp over the whole cut, and a dense case against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def single_term_case(n=4096, sigma=0.01, x0=30.0, seed=0):
    # samples 1 ER apart (the 6 sigma cut is 0.06 ER), one ray near each at a
    # distance from 0 to just inside the cut, so that F_k holds one Gaussian
    rng = np.random.default_rng(seed)
    s = np.column_stack([x0 + np.arange(n, dtype=np.float64), np.full(n, 5.0)])
    r = np.linspace(0.0, 5.999 * sigma, n)
    rng.shuffle(r)
    t = rng.uniform(0, 2 * np.pi, n)
    y = s + np.column_stack([r * np.cos(t), r * np.sin(t)])
    d = y - s
    G = np.exp(-(d[:, 0] ** 2 + d[:, 1] ** 2) / (2 * sigma ** 2))
    return s, y, d, G


@pytest.mark.parametrize("x0", [0.0, 30.0, -1000.0])
def test_single_gaussians_match_float64_exp(x0):
    sigma, w = 0.01, 1e-4
    s, y, d, G = single_term_case(x0=x0)
    norm = w / (2 * np.pi * sigma ** 2)
    F = lens.light_curve(T(y), w, T(s), sigma).cpu().numpy()
    # float-float: ~2^-47 per operation; the exponent reaches -18 at the cut
    np.testing.assert_allclose(F, norm * G, rtol=2e-13, atol=0)
    # the gradient of L = sum_k F_k^2 (T = 0): dL/dy = 2 F_k norm G (-(y - s) / sigma^2)
    gy = lens.light_curve_grad(T(y), w, T(s), sigma, T(F), T(np.zeros_like(F))).cpu().numpy()
    ref = (2 * F * norm * G / sigma ** 2)[:, None] * (-d)
    np.testing.assert_allclose(gy, ref, rtol=2e-12, atol=1e-12 * np.abs(ref).max())


def test_rays_beyond_the_cut_and_on_a_sample():
    sigma, w = 0.02, 1.0
    s = np.array([[0.0, 0.0], [10.0, 0.0], [20.0, 0.0]])
    # exactly on the first sample, 6.001 sigma from the second (out), two
    # rays 3 sigma from the third
    y = np.array([[0.0, 0.0], [10.0 + 6.001 * sigma, 0.0], [20.0, 3 * sigma], [20.0, -3 * sigma]])
    F = lens.light_curve(T(y), w, T(s), sigma).cpu().numpy()
    norm = w / (2 * np.pi * sigma ** 2)
    np.testing.assert_allclose(F, [norm, 0.0, 2 * norm * np.exp(-4.5)], rtol=1e-13, atol=0)
    ref = oracle.light_curve(y, w, s, sigma)
    np.testing.assert_allclose(F, ref, rtol=1e-13, atol=0)


def test_dense_light_curve_and_gradient_match_oracle():
    rng = np.random.default_rng(3)
    y = rng.uniform(-1.0, 1.0, (40000, 2)) + np.array([12.0, -3.0])
    t = np.linspace(-0.9, 0.9, 300)
    s = np.column_stack([12.0 + t, -3.0 + 0.5 * t])
    sigma, w = 0.05, 1e-4
    F = lens.light_curve(T(y), w, T(s), sigma).cpu().numpy()
    F_o = oracle.light_curve(y, w, s, sigma)
    np.testing.assert_allclose(F, F_o, rtol=1e-12, atol=1e-14 * np.abs(F_o).max())
    Tk = 0.9 * F_o
    g = lens.light_curve_grad(T(y), w, T(s), sigma, T(F), T(Tk)).cpu().numpy()
    g_o = oracle.light_curve_grad(y, w, s, sigma, F_o, Tk)
    np.testing.assert_allclose(g, g_o, rtol=1e-9, atol=1e-12 * np.abs(g_o).max())
