"""Images of a point source and the lensed image of a Gaussian source on a
deflected grid (Sec. 2.5), through the C-ABI against the oracle on the same
deflections: the image cells must be the same cells; where the oracle's
Newton inversion has converged, positions agree to 1e-12 and inverse
magnifications (det of the lens map's Jacobian, O(1) away from masses) to
1e-10 or 1e-9 relative (the two
sides differ only by the rounding of the Newton steps)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens, synth

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def residual(y, g, cell, x1, x2, beta):
    """|p(s, t) - beta| of the cell's bilinear map at the reported point."""
    nx = y.shape[1] - 1
    j, i = divmod(int(cell), nx)
    s, t = (x1 - g.x0) / g.h - i, (x2 - g.y0) / g.h - j
    q0, q1, q2, q3 = y[j, i], y[j, i + 1], y[j + 1, i + 1], y[j + 1, i]
    p = q0 + s * (q1 - q0) + t * (q3 - q0) + s * t * (q0 - q1 + q2 - q3)
    return float(np.hypot(*(p - np.asarray(beta))))


def check_parity(y, g, beta):
    cells, imgs = lens.find_images(T(y), g, beta)
    cells, imgs = cells.cpu().numpy(), imgs.cpu().numpy()
    ref = oracle.find_images(y, g.x0, g.y0, g.h, beta)
    assert cells.tolist() == [r[0] for r in ref]
    n_conv = 0
    for k, (c, x1, x2, mu) in enumerate(ref):
        if residual(y, g, c, x1, x2, beta) < 1e-12 * (1 + np.abs(y).max()):
            n_conv += 1
            assert imgs[k, 0] == pytest.approx(x1, abs=1e-12)
            assert imgs[k, 1] == pytest.approx(x2, abs=1e-12)
            assert 1.0 / imgs[k, 2] == pytest.approx(1.0 / mu, rel=1e-9, abs=1e-10)
    return ref, n_conv


def test_point_lens_images_and_closed_form():
    beta = (0.2, -0.1)
    g = synth.Grid(x0=-1.6 + 1e-4 * np.pi, y0=-1.6 + 1e-4 * np.e, h=0.004, nx=800, ny=800)
    with lens.LensFMM(T(np.zeros((1, 2))), T(np.ones(1)), 0.0, 0.0, p=40, leaf_size=8,
                      prec=lens.FP64, target_box=(g.x0, g.x0 + 3.2, g.y0, g.y0 + 3.2)) as P:
        y = P.deflect_grid(g).cpu().numpy()
    ref, n_conv = check_parity(y, g, beta)
    big = [r for r in ref if abs(r[3]) >= 1e-6]
    assert len(big) == 2 and n_conv >= 2
    # a one-slot buffer: the binding calls again with the reported count
    cells, imgs = lens.find_images(T(y), g, beta, max_out=1)
    assert cells.cpu().tolist() == [r[0] for r in ref]
    u = np.hypot(*beta)
    tot = (u * u + 2) / (u * np.sqrt(u * u + 4))
    assert sum(abs(r[3]) for r in big) == pytest.approx(tot, rel=1.5e-2)


@pytest.mark.parametrize("prec", [lens.FP64, lens.FP32_BULK])
def test_star_field_images(prec):
    f = synth.config_uniform(seed=4, n=400, kappa_star=0.3, kappa_s=0.1, gamma=0.2)
    g = synth.Grid(x0=-3.0, y0=-3.0, h=0.01, nx=600, ny=600)
    box = (g.x0, g.x0 + g.nx * g.h, g.y0, g.y0 + g.ny * g.h)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=24, leaf_size=8, prec=prec,
                      target_box=box) as P:
        y = P.deflect_grid(g).cpu().numpy()
    rng = np.random.default_rng(5)
    total = 0
    for beta in rng.uniform(-1.0, 1.0, size=(6, 2)):
        ref, n_conv = check_parity(y, g, tuple(beta))
        total += len(ref)
    assert total >= 6


def test_halo_images():
    # elliptical NFW stand-in (2e6 equal-mass particles), 1024^2 cells over
    # +-2 r_s, float32-bulk deflections: the image cells of sources near the
    # centre, including the particles' own demagnified images
    f = synth.nfw_halo(seed=1, n=2_000_000, grid_n=1025)
    g = f.grid
    box = (g.x0, g.x0 + g.nx * g.h, g.y0, g.y0 + g.ny * g.h)
    with lens.LensFMM(T(f.stars), T(f.masses), 0.0, 0.0, p=16, leaf_size=16,
                      prec=lens.FP32_BULK, target_box=box) as P:
        yd = P.deflect_grid(g)
    y = yd.cpu().numpy()
    found = 0
    for beta in [(0.031, -0.017), (0.2, 0.1), (-0.4, 0.05)]:
        ref, n_conv = check_parity(y, g, beta)
        found += len(ref)
        print("halo, beta %s: %d image cells (%d converged), mu %s"
              % (beta, len(ref), n_conv, ["%.3g" % r[3] for r in ref][:8]))
    assert found >= 3


def test_no_image_far_away_and_source_image():
    f = synth.config_uniform(seed=6, n=200, kappa_star=0.3, kappa_s=0.0, gamma=0.1)
    g = synth.Grid(x0=-2.0, y0=-2.0, h=0.02, nx=200, ny=200)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=24, leaf_size=8,
                      prec=lens.FP64, target_box=(-2.0, 2.0, -2.0, 2.0)) as P:
        yd = P.deflect_grid(g)
    cells, imgs = lens.find_images(yd, g, (500.0, 500.0))
    assert cells.shape[0] == 0 and imgs.shape == (0, 3)
    beta, sig = (0.1, -0.05), 0.05
    img = lens.source_image(yd, beta, sig)
    assert img.shape == yd.shape[:2]
    ref = oracle.source_image(yd.cpu().numpy(), beta, sig).reshape(img.shape)
    # the exponent reaches ~745 before underflow: one rounding of it moves the
    # value by up to ~745 * 2^-53 = 8e-14 relative
    np.testing.assert_allclose(img.cpu().numpy(), ref, rtol=5e-13, atol=1e-300)


def test_nan_corner_matches_oracle():
    # identity lens on a 6 x 6 corner grid, the source inside cell (2, 2);
    # with that cell's top-left corner undefined the oracle finds no image
    # there, and neither may the kernel (which must not build the bounding
    # box from the three finite corners)
    g = synth.Grid(x0=0.0, y0=0.0, h=1.0, nx=5, ny=5)
    y = g.corners().copy()
    beta = (2.5, 2.5)
    assert [r[0] for r in oracle.find_images(y, g.x0, g.y0, g.h, beta)] == [12]
    y[3, 2] = (np.nan, 3.0)
    ref, _ = check_parity(y, g, beta)
    assert ref == []
    y[3, 2] = (2.0, np.nan)
    ref, _ = check_parity(y, g, beta)
    assert ref == []
