"""Map consumers (finite Gaussian source, histogram, track) on the GPU against
the oracle's, on a real map and on the pinned synthetic cases."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens, synth

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def c1_map():
    f = synth.c1_plain(seed=0)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=24, leaf_size=16,
                      prec=lens.FP32_BULK, target_box=(-10, 10, -10, 10)) as P:
        mp, _ = P.ipm_map(f.grid, f.box, f.npx, f.npy)
    return f, mp.cpu().numpy()


@pytest.mark.parametrize("sigma,trunc", [(0.7, 6.0), (2.5, 4.0), (6.0, 3.0)])
def test_finite_source_matches_oracle(c1_map, sigma, trunc):
    f, mp = c1_map
    out = lens.map_source(T(mp), sigma, trunc).cpu().numpy()
    ref = oracle.map_convolve_gaussian(mp, sigma, trunc)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_finite_source_of_a_constant_and_a_point():
    mp = np.full((50, 70), 2.5)
    # the weighted sums run in float-float (~48 bits): a few hundred terms
    # keep ~1e-13 of the float64 normalisation
    np.testing.assert_allclose(lens.map_source(T(mp), 3.0).cpu().numpy(), 2.5, rtol=2e-13)
    pt = np.zeros((61, 61))
    pt[30, 30] = 1.0
    out = lens.map_source(T(pt), 2.0).cpu().numpy()
    np.testing.assert_allclose(out, oracle.map_convolve_gaussian(pt, 2.0), rtol=1e-12,
                               atol=1e-18)


@pytest.mark.parametrize("log_bins", [False, True])
def test_histogram_matches_oracle(c1_map, log_bins):
    f, mp = c1_map
    lo, hi = (-0.5, 1.5) if log_bins else (0.0, 12.0)
    c = lens.map_histogram(T(mp), lo, hi, 64, log_bins=log_bins).cpu().numpy()
    ref = oracle.histogram(mp, lo, hi, 64, log_bins=log_bins)
    assert c.sum() == mp.size == ref.sum()
    # log10 may differ by an ulp between libraries: a value on a bin edge may
    # move to the neighbouring bin
    assert np.abs(c - ref).max() <= (2 if log_bins else 0)


def test_track_matches_oracle(c1_map):
    f, mp = c1_map
    t = np.linspace(-4.8, 4.8, 2048)
    s = np.column_stack([t * np.cos(0.5), t * np.sin(0.5)])
    out = lens.map_track(T(mp), f.box, T(s)).cpu().numpy()
    np.testing.assert_allclose(out, oracle.map_track(mp, f.box, s), rtol=1e-13)


def test_light_curve_of_a_finite_source_from_the_map(c1_map):
    # the paper's use: the map seen by a finite source, sampled along a track
    f, mp = c1_map
    src = lens.map_source(T(mp), 1.5)
    t = np.linspace(-4.0, 4.0, 500)
    s = np.column_stack([t, 0.3 * t])
    lc = lens.map_track(src, f.box, T(s)).cpu().numpy()
    ref = oracle.map_track(oracle.map_convolve_gaussian(mp, 1.5), f.box, s)
    np.testing.assert_allclose(lc, ref, rtol=1e-11)
    assert np.all(lc > 0)
