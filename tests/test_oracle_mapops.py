"""Pins of the oracle's map consumers (Sec. 3: finite-source magnification
histograms and light curves from a map): closed forms and library routines."""
import numpy as np
import pytest

import oracle


def test_gaussian_source_keeps_a_constant_map():
    mp = np.full((20, 30), 3.25)
    np.testing.assert_allclose(oracle.map_convolve_gaussian(mp, 2.3), 3.25, rtol=1e-14)


def test_gaussian_source_of_a_point_is_the_normalised_kernel():
    mp = np.zeros((61, 61))
    mp[30, 30] = 1.0
    s = 2.0
    out = oracle.map_convolve_gaussian(mp, s, trunc=6.0)
    # where the kernel around p lies inside the map: out[p] = w(p - c) / sum(w)
    d = np.arange(-12, 13)
    w1 = np.exp(-d * d / (2 * s * s))
    W = np.outer(w1, w1)
    ref = W / W.sum()
    np.testing.assert_allclose(out[18:43, 18:43], ref, rtol=1e-12, atol=1e-16)


def test_gaussian_source_of_a_linear_map_in_the_interior():
    # a symmetric kernel leaves a linear function unchanged away from the edges
    y, x = np.mgrid[0:40, 0:50]
    mp = 1.0 + 0.5 * x - 0.25 * y
    out = oracle.map_convolve_gaussian(mp, 1.5, trunc=4.0)
    np.testing.assert_allclose(out[8:-8, 8:-8], mp[8:-8, 8:-8], rtol=1e-13)


def test_histogram_matches_numpy():
    rng = np.random.default_rng(0)
    v = rng.lognormal(0.5, 1.0, 10000)
    lo, hi, nb = -1.0, 2.0, 30
    c = oracle.histogram(v, lo, hi, nb, log_bins=True)
    ref, _ = np.histogram(np.log10(v), bins=nb, range=(lo, hi))
    np.testing.assert_array_equal(c[1:-1], ref)
    assert c[0] == np.sum(np.log10(v) < lo) and c[-1] == np.sum(np.log10(v) >= hi)
    assert c.sum() == v.size
    lin = oracle.histogram(v, 0.0, 10.0, 20)
    ref2, _ = np.histogram(v, bins=20, range=(0.0, 10.0))
    np.testing.assert_array_equal(lin[1:-1], ref2)


def test_track_is_exact_on_a_bilinear_map():
    box = (-2.0, 2.0, -1.0, 1.0)
    npx, npy = 40, 20
    cx = box[0] + (np.arange(npx) + 0.5) * 0.1
    cy = box[2] + (np.arange(npy) + 0.5) * 0.1
    X, Y = np.meshgrid(cx, cy)
    mp = 2.0 + 0.3 * X - 0.7 * Y + 0.05 * X * Y
    rng = np.random.default_rng(1)
    s = np.column_stack([rng.uniform(cx[0], cx[-1], 500), rng.uniform(cy[0], cy[-1], 500)])
    out = oracle.map_track(mp, box, s)
    ref = 2.0 + 0.3 * s[:, 0] - 0.7 * s[:, 1] + 0.05 * s[:, 0] * s[:, 1]
    np.testing.assert_allclose(out, ref, rtol=1e-12)
    # at a pixel centre the value is the pixel's
    assert oracle.map_track(mp, box, np.array([[cx[7], cy[3]]]))[0] == pytest.approx(mp[3, 7])
