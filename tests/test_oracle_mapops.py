"""Pins of the oracle's map consumers (Sec. 3: finite-source magnification
histograms and light curves from a map): closed forms and library routines."""
import numpy as np
import pytest

import oracle


def test_gaussian_source_keeps_a_constant_map():
    mp = np.full((20, 30), 3.25)
    np.testing.assert_allclose(oracle.map_convolve_gaussian(mp, 2.3), 3.25, rtol=1e-14)


def test_gaussian_source_of_a_point_is_the_kernel_cut_at_the_isophote():
    # a point map shows the window: nonzero exactly on the disk |d| <= trunc
    # sigma (the source profile cut at an isophote), shaped like
    # exp(-|d|^2 / 2 sigma^2) inside it
    mp = np.zeros((61, 61))
    mp[30, 30] = 1.0
    s, trunc = 2.0, 3.3  # radius 6.6 pixels
    out = oracle.map_convolve_gaussian(mp, s, trunc=trunc)
    d = np.arange(-30, 31)
    r2 = d[None, :] ** 2 + d[:, None] ** 2
    inside = r2 <= (trunc * s) ** 2
    assert np.all(out[inside] > 0) and np.all(out[~inside] == 0)
    # e.g. (4, 5) is inside (41 <= 43.56), (5, 5) outside, on a 12-pixel square
    assert out[34, 35] > 0 and out[35, 35] == 0
    ratio = out[inside] / out[30, 30]
    np.testing.assert_allclose(ratio, np.exp(-r2[inside] / (2 * s * s)), rtol=1e-13)


def test_gaussian_source_normalisation_is_the_untruncated_integral():
    # far from the edges with a long tail, sum_k exp(-|k|^2 / 2 s^2) over the
    # integer lattice is 2 pi s^2 up to exp(-2 pi^2 s^2) (Poisson summation),
    # so the point map's peak is 1 / (2 pi s^2)
    mp = np.zeros((61, 61))
    mp[30, 30] = 1.0
    for s in (2.0, 2.4):
        out = oracle.map_convolve_gaussian(mp, s, trunc=12.0)
        assert out[30, 30] * 2 * np.pi * s * s == pytest.approx(1.0, rel=1e-13)


def test_gaussian_source_of_a_quadratic_map_converges_to_the_exact_convolution():
    # the untruncated Gaussian convolution of a quadratic f is
    # f + sigma^2 (f_xx + f_yy) / 2 (lattice second moment sigma^2 up to
    # exp(-2 pi^2 sigma^2)); the truncated, renormalised source approaches it
    # as the cut moves out, the error falling like the profile's tail
    y, x = np.mgrid[0:80, 0:90].astype(float)
    a, b, c = 0.3, -0.1, 0.05
    f = a * (x - 40) ** 2 + b * (y - 35) ** 2 + c * (x - 40) * (y - 35) + 0.2 * x - 0.7 * y + 3
    s = 1.5
    exact = f + (a + b) * s * s
    inner = (slice(20, -20), slice(20, -20))
    errs = [np.abs(oracle.map_convolve_gaussian(f, s, trunc=t)[inner] - exact[inner]).max()
            for t in (3.0, 4.0, 5.0, 6.0, 8.0)]
    assert all(e1 < 0.2 * e0 for e0, e1 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-11


def test_gaussian_source_second_moment_is_the_disk_cut_profiles():
    # the window's second moment, read off the map (x - x0)^2: for a Gaussian
    # cut at radius T sigma, E[dx^2] = sigma^2 (1 - (T^2/2) e^{-T^2/2} /
    # (1 - e^{-T^2/2})) (continuous; the lattice adds ~0.2% at sigma = 6 px),
    # which a square cut at +-T sigma would put at 0.973 sigma^2 for T = 3
    s, T = 6.0, 3.0
    yy, xx = np.mgrid[0:101, 0:101].astype(float)
    out = oracle.map_convolve_gaussian((xx - 50.0) ** 2, s, trunc=T)
    disk = 1 - (T * T / 2) * np.exp(-T * T / 2) / (1 - np.exp(-T * T / 2))
    assert out[50, 50] / s ** 2 == pytest.approx(disk, rel=4e-3)


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
