"""Pins of the oracle's image finder and Gaussian-source image (Sec. 2.5)
against closed forms: the single image of an affine lens, the two images of
a point lens (positions, magnifications, the total magnification of the
point lens), and the lens equation evaluated at the returned positions."""
import numpy as np
import pytest

import oracle
from paper_2211_00354_gb300 import synth


def affine_grid_y(kappa, gamma, grid):
    x = grid.corners()
    return np.stack([(1 - kappa - gamma) * x[..., 0], (1 - kappa + gamma) * x[..., 1]], axis=-1)


@pytest.mark.parametrize("kappa,gamma", [(0.3, 0.2), (0.5, 0.8), (1.4, 0.1)])
def test_affine_lens_single_image(kappa, gamma):
    # y = A x with A = diag(a, b): one image at A^-1 beta with mu = 1/(a b),
    # negative when a and b differ in sign; the bilinear map is exact
    g = synth.Grid(x0=-2.013, y0=-1.987, h=0.05, nx=80, ny=80)
    y = affine_grid_y(kappa, gamma, g)
    a, b = 1 - kappa - gamma, 1 - kappa + gamma
    beta = (0.1234 * a, -0.0567 * b)
    imgs = oracle.find_images(y, g.x0, g.y0, g.h, beta)
    assert len(imgs) == 1
    _, x1, x2, mu = imgs[0]
    assert x1 == pytest.approx(0.1234, abs=1e-12)
    assert x2 == pytest.approx(-0.0567, abs=1e-12)
    assert mu == pytest.approx(1.0 / (a * b), rel=1e-12)


def point_lens_case(beta, h=0.004):
    g = synth.Grid(x0=-1.6 + 1e-4 * np.pi, y0=-1.6 + 1e-4 * np.e, h=h, nx=int(3.2 / h), ny=int(3.2 / h))
    y = oracle.deflect(np.zeros((1, 2)), np.ones(1), 0.0, 0.0, g.corners().reshape(-1, 2))
    return g, y.reshape(g.ny + 1, g.nx + 1, 2)


def point_lens_images(beta, h=0.004):
    g, y = point_lens_case(beta, h)
    return g, oracle.find_images(y, g.x0, g.y0, g.h, beta)


@pytest.mark.parametrize("beta", [(0.2, -0.1), (-0.35, 0.5)])
def test_point_lens_two_images(beta):
    g, imgs = point_lens_images(beta)
    # the cell holding the mass maps to a polygon around everything near it:
    # it reports the mass's infinitely demagnified image (mu ~ h^2 / inf)
    core = [im for im in imgs if abs(im[3]) < 1e-6]
    imgs = [im for im in imgs if abs(im[3]) >= 1e-6]
    assert len(imgs) == 2 and len(core) <= 1
    for _, x1, x2, mu in core:
        assert np.hypot(x1, x2) < 2 * g.h
    u = np.hypot(*beta)
    bhat = np.asarray(beta) / u
    xs = {1: (u + np.sqrt(u * u + 4)) / 2, -1: (u - np.sqrt(u * u + 4)) / 2}
    total = 0.0
    for _, x1, x2, mu in imgs:
        par = 1 if mu > 0 else -1
        xe = xs[par] * bhat
        # bilinear cells: positions to O(h^2); the Jacobian of the bilinear
        # map away from the cell centre is a one-sided difference, so the
        # magnification is first order in h (see the convergence test)
        assert np.hypot(x1 - xe[0], x2 - xe[1]) < 5e-5
        assert mu == pytest.approx(1.0 / (1.0 - xs[par] ** -4), rel=1.5e-2)
        total += abs(mu)
        # the lens equation at the returned position gives back beta
        r2 = x1 * x1 + x2 * x2
        assert np.hypot(x1 - x1 / r2 - beta[0], x2 - x2 / r2 - beta[1]) < 5e-5
    # total magnification of a point lens, (u^2 + 2) / (u sqrt(u^2 + 4))
    assert total == pytest.approx((u * u + 2) / (u * np.sqrt(u * u + 4)), rel=1.5e-2)


def test_point_lens_magnification_converges_first_order():
    beta = (0.2, -0.1)
    u = np.hypot(*beta)
    exact = {1: 1.0 / (1.0 - ((u + np.sqrt(u * u + 4)) / 2) ** -4),
             -1: 1.0 / (1.0 - ((u - np.sqrt(u * u + 4)) / 2) ** -4)}
    errs = []
    for h in (0.004, 0.002):
        _, imgs = point_lens_images(beta, h)
        imgs = [im for im in imgs if abs(im[3]) >= 1e-6]
        errs.append(max(abs(mu / exact[1 if mu > 0 else -1] - 1) for *_, mu in imgs))
    assert errs[1] < 0.7 * errs[0]


def test_winding_and_bounding_box():
    # a unit square cell and its reflection: winding +1 and -1 inside, 0 on
    # the far side of each half-open edge and outside the bounding box
    y = np.array([[[0.0, 0.0], [1.0, 0.0]], [[0.0, 1.0], [1.0, 1.0]]])
    assert oracle.winding_numbers(y, (0.5, 0.5))[0, 0] == 1
    assert oracle.winding_numbers(y[:, ::-1], (0.5, 0.5))[0, 0] == -1
    assert oracle.winding_numbers(y, (0.5, 1.0))[0, 0] == 0   # top edge: half-open
    assert oracle.winding_numbers(y, (0.5, 0.0))[0, 0] == 1   # bottom edge counts
    assert oracle.winding_numbers(y, (1.5, 0.5))[0, 0] == 0
    # neighbouring cells share edges: a point on the shared edge belongs to one
    y2 = np.array([[[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]], [[0.0, 1.0], [1.0, 1.0], [2.0, 1.0]]])
    w = oracle.winding_numbers(y2, (1.0, 0.5))
    assert int(np.abs(w).sum()) == 1


def test_a_nan_corner_holds_no_image():
    # an undefined corner leaves the cell's bounding box undefined: no image,
    # even where the remaining edges would wind around the source (here the
    # right edge, upward with beta on its left, alone would give +1)
    y = np.array([[[0.0, 0.0], [1.0, 0.0]], [[np.nan, 1.0], [1.0, 1.0]]])
    assert oracle.winding_numbers(y, (0.5, 0.5))[0, 0] == 0
    y[1, 0] = (0.0, 1.0)
    assert oracle.winding_numbers(y, (0.5, 0.5))[0, 0] == 1


def test_source_image_closed_form():
    beta, sig = (0.3, -0.2), 0.05
    y = np.array([[0.3, -0.2], [0.35, -0.2], [0.3, -0.1], [10.0, 10.0]])
    v = oracle.source_image(y, beta, sig)
    assert v[0] == 1.0
    assert v[1] == pytest.approx(np.exp(-0.5), rel=1e-14)
    assert v[2] == pytest.approx(np.exp(-2.0), rel=1e-14)
    assert v[3] == 0.0
