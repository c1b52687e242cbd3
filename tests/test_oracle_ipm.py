"""Pins of the oracle's first-order IPM (Sec. 2.3; step 4 of Sec. 2.4).

The overlap routine is pinned by hand-computed cases (tests/golden) and by an
independent second route (Green's theorem edge integration) plus point
sampling; the map is pinned by exact results (an affine lens magnifies every
pixel by 1/|det A|), the point-lens magnification (u^2+2)/(u sqrt(u^2+4)),
the flux ledger and brute force on tiny inputs.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2211_00354_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "clip_cases.txt")


def golden_cases():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, poly = line.split("|")
        px, py, exp = head.split()
        v = np.array([float(t) for t in poly.split()]).reshape(-1, 2)
        out.append((int(px), int(py), float(exp), v))
    return out


@pytest.mark.parametrize("case", golden_cases())
def test_clip_golden(case):
    px, py, exp, v = case
    assert oracle.clip_area_sh(v, px, py) == pytest.approx(exp, abs=1e-14)
    assert oracle.clip_area_green(v, px, py) == pytest.approx(exp, abs=1e-14)


def random_quads(rng, n, spread=1.5):
    c = rng.uniform(-1, 2, (n, 1, 2))
    return c + rng.normal(0, spread, (n, 4, 2)) * rng.uniform(0.05, 1, (n, 1, 1))


def test_two_clip_routes_agree():
    rng = np.random.default_rng(0)
    for q in random_quads(rng, 400):
        for px, py in [(0, 0), (1, 0), (-1, 1), (1, 1)]:
            a = oracle.clip_area_sh(q, px, py)
            b = oracle.clip_area_green(q, px, py)
            assert a == pytest.approx(b, abs=1e-12)


def winding_number(poly, pts):
    # crossing-number with orientation (independent of both clip routines)
    w = np.zeros(len(pts))
    n = len(poly)
    for k in range(n):
        a, b = poly[k], poly[(k + 1) % n]
        up = (a[1] <= pts[:, 1]) & (b[1] > pts[:, 1])
        dn = (a[1] > pts[:, 1]) & (b[1] <= pts[:, 1])
        cross = (b[0] - a[0]) * (pts[:, 1] - a[1]) - (pts[:, 0] - a[0]) * (b[1] - a[1])
        w += np.where(up & (cross > 0), 1, 0) - np.where(dn & (cross < 0), 1, 0)
    return w


def test_clip_matches_point_sampling():
    rng = np.random.default_rng(1)
    s = (np.arange(400) + 0.5) / 400
    X, Y = np.meshgrid(s, s)
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    for q in random_quads(rng, 25, spread=0.8):
        est = winding_number(q, pts).mean()
        assert oracle.clip_area_sh(q, 0, 0) == pytest.approx(est, abs=4e-3)


def test_pixel_areas_sum_to_shoelace():
    rng = np.random.default_rng(2)
    for q in random_quads(rng, 50, spread=1.0):
        tot = sum(oracle.clip_area_sh(q, px, py) for px in range(-8, 9) for py in range(-8, 9))
        x, y = q[:, 0], q[:, 1]
        sl = 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
        if np.abs(q).max() < 7.5:
            assert tot == pytest.approx(sl, abs=1e-12)


def affine_corners(grid, a, b, c=0.0):
    xc = grid.corners()
    y = np.empty_like(xc)
    y[..., 0] = a * xc[..., 0] + c * xc[..., 1]
    y[..., 1] = c * xc[..., 0] + b * xc[..., 1]
    return y


@pytest.mark.parametrize("a,b,c", [(1.0, 1.0, 0.0), (0.55, 1.45, 0.0), (-0.3, 0.8, 0.1), (0.2, -0.6, 0.05)])
def test_affine_lens_gives_inverse_determinant(a, b, c):
    # a linear lens map y = A x sends each cell to a parallelogram of area
    # |det A| h^2, so every fully covered pixel has mu = 1/|det A| exactly.
    grid = synth.Grid(x0=-12.0, y0=-12.0, h=0.173, nx=139, ny=139)
    y = affine_corners(grid, a, b, c)
    box = (-1.0, 1.0, -1.5, 0.5)
    mp, st = oracle.ipm_map(y, grid.h, box, 16, 12)
    det = a * b - c * c
    np.testing.assert_allclose(mp, 1.0 / abs(det), rtol=1e-10)
    led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
    assert led == pytest.approx(st["area_total"], rel=1e-12)
    assert np.sum(mp) * (2.0 / 16) * (2.0 / 12) == pytest.approx(st["area_in_map"], rel=1e-12)


def point_lens_pixel_mu(box, npx, npy, nq=8):
    # (u^2+2)/(u sqrt(u^2+4)) averaged over each pixel by Gauss-Legendre
    g, w = np.polynomial.legendre.leggauss(nq)
    du = (box[1] - box[0]) / npx
    dv = (box[3] - box[2]) / npy
    out = np.zeros((npy, npx))
    for j in range(npy):
        for i in range(npx):
            u = box[0] + (i + 0.5 + 0.5 * g) * du
            v = box[2] + (j + 0.5 + 0.5 * g) * dv
            U, V = np.meshgrid(u, v)
            r = np.hypot(U, V)
            mu = (r * r + 2) / (r * np.sqrt(r * r + 4))
            out[j, i] = np.sum(w[None, :] * w[:, None] * mu) / 4.0
    return out


def test_point_lens_magnification_map():
    # m = 1 at the origin, no smooth field; n_0 = (du/h)^2 = 16 rays per pixel
    box = (-2.0, 2.0, -2.0, 2.0)
    npx = npy = 40
    h = 0.025
    grid = synth.Grid(x0=-3.5 + 0.5 * h, y0=-3.5 + 0.5 * h, h=h, nx=280, ny=280)
    xc = grid.corners().reshape(-1, 2)
    y = oracle.deflect(np.zeros((1, 2)), [1.0], 0.0, 0.0, xc).reshape(grid.ny + 1, grid.nx + 1, 2)
    mp, st = oracle.ipm_map(y, grid.h, box, npx, npy, bbox_cap=64)
    ref = point_lens_pixel_mu(box, npx, npy)
    cu = box[0] + (np.arange(npx) + 0.5) * 0.1
    U, V = np.meshgrid(cu, cu)
    far = np.hypot(U, V) - 0.075 >= 0.2
    rel = np.abs(mp[far] - ref[far]) / ref[far]
    assert rel.mean() < 1e-3, rel.mean()
    led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
    assert led == pytest.approx(st["area_total"], rel=1e-12)


def test_tiny_brute_force_rasterisation():
    # 4 x 4 cells, 8 x 8 map: compare with point-sampled winding numbers
    rng = np.random.default_rng(5)
    grid = synth.Grid(x0=0.0, y0=0.0, h=1.0, nx=4, ny=4)
    xc = grid.corners()
    y = xc * 0.9 + rng.normal(0, 0.12, xc.shape) + 0.2
    box = (0.0, 4.0, 0.0, 4.0)
    mp, st = oracle.ipm_map(y, grid.h, box, 8, 8)
    s = (np.arange(160) + 0.5) / 160 * 0.5
    brute = np.zeros((8, 8))
    for j in range(4):
        for i in range(4):
            poly = np.array([y[j, i], y[j, i + 1], y[j + 1, i + 1], y[j + 1, i]])
            x_, y_ = poly[:, 0], poly[:, 1]
            AP = 0.5 * np.sum(x_ * np.roll(y_, -1) - np.roll(x_, -1) * y_)
            for py in range(8):
                for px in range(8):
                    X, Y = np.meshgrid(px * 0.5 + s, py * 0.5 + s)
                    wn = winding_number(poly, np.stack([X.ravel(), Y.ravel()], 1)).mean() * 0.25
                    brute[py, px] += grid.h ** 2 * wn / AP / 0.25
    np.testing.assert_allclose(mp, brute, atol=2e-2 * np.abs(brute).max())


def test_mean_magnification_of_random_field():
    # <mu> -> 1/|(1-kappa)^2 - gamma^2| on large maps (statistical).  The exact
    # form of this invariant is the affine-lens test above; here an ensemble of
    # 8 seeded fields (kappa_* = 0.1 in stars, kappa_s = 0.3, gamma = 0.2)
    # must reproduce it within 10%.
    kappa, gamma = 0.4, 0.2
    mu_th = 1.0 / abs((1 - kappa) ** 2 - gamma ** 2)
    vals = []
    for seed in range(8):
        f = synth.config_uniform(seed=seed, n=3000, kappa_star=0.1, kappa_s=0.3, gamma=gamma)
        grid = synth.shooting_grid(kappa, gamma, 6.0, 0.08, margin_frac=0.5)
        y = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, grid.corners().reshape(-1, 2))
        y = y.reshape(grid.ny + 1, grid.nx + 1, 2)
        mp, st = oracle.ipm_map(y, grid.h, (-6, 6, -6, 6), 24, 24, bbox_cap=64)
        vals.append(mp[3:-3, 3:-3].mean() / mu_th)
        led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
        assert led == pytest.approx(st["area_total"], rel=1e-12)
    assert abs(np.mean(vals) - 1) < 0.10, vals


# ---- refinement of cells larger than the cap (2 x 2 split, new corner rays) --

def _corner_grid(stars, masses, ks, g, grid):
    xc = grid.corners().reshape(-1, 2)
    return oracle.deflect(stars, masses, ks, g, xc).reshape(grid.ny + 1, grid.nx + 1, 2)


def test_refinement_with_no_levels_is_the_plain_map():
    f = synth.config_uniform(seed=3, n=40, kappa_star=0.3, kappa_s=0.1, gamma=0.2)
    grid = synth.Grid(x0=-3.0, y0=-3.0, h=0.25, nx=24, ny=24)
    y = _corner_grid(f.stars, f.masses, f.kappa_s, f.gamma, grid)
    box = (-2.0, 2.0, -2.0, 2.0)
    mp, st = oracle.ipm_map(y, grid.h, box, 30, 30, bbox_cap=3)
    mr, sr = oracle.ipm_map_refined(y, grid.x0, grid.y0, grid.h, f.stars, f.masses, f.kappa_s,
                                    f.gamma, box, 30, 30, 3, 0)
    assert np.array_equal(mp, mr) and st == sr
    assert st["cells_dropped"] > 0


def test_refined_affine_map_equals_the_uncapped_map():
    # an affine lens (one massless star): the four sub-cells of a cell tile its
    # image exactly, so splitting the cells a cap rejects gives the map every
    # cell would give uncapped
    star, m = np.array([[0.3, -0.2]]), np.array([0.0])
    ks, g = -2.0, 0.5  # y = diag(2.5, 3.5) x: cells grow ~3x
    grid = synth.Grid(x0=-0.5, y0=-0.4, h=0.1, nx=10, ny=8)
    y = _corner_grid(star, m, ks, g, grid)
    box = (-1.5, 1.5, -1.5, 1.5)
    full, sf = oracle.ipm_map(y, grid.h, box, 30, 30, bbox_cap=0)
    capped, sc = oracle.ipm_map(y, grid.h, box, 30, 30, bbox_cap=4)
    ref, sr = oracle.ipm_map_refined(y, grid.x0, grid.y0, grid.h, star, m, ks, g, box, 30, 30, 4, 3)
    assert sc["cells_dropped"] > 0 and sr["cells_dropped"] == 0
    np.testing.assert_allclose(ref, full, rtol=1e-12, atol=1e-12)
    assert sr["area_in_map"] == pytest.approx(sf["area_in_map"], rel=1e-12)
    assert not np.allclose(capped, full)


def test_refinement_recovers_flux_near_a_point_lens():
    # cells next to the lens map to huge polygons: each level splits what the
    # cap rejects, the dropped area falls and the ledger stays closed
    box = (-2.0, 2.0, -2.0, 2.0)
    h = 0.05
    grid = synth.Grid(x0=-2.0 + 0.5 * h, y0=-2.0 + 0.3 * h, h=h, nx=80, ny=80)
    star, m = np.zeros((1, 2)), np.array([1.0])
    y = _corner_grid(star, m, 0.0, 0.0, grid)
    dropped = []
    for levels in (0, 1, 2, 3):
        mp, st = oracle.ipm_map_refined(y, grid.x0, grid.y0, grid.h, star, m, 0.0, 0.0, box, 40,
                                        40, 8, levels)
        led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
        assert led == pytest.approx(st["area_total"], rel=1e-12)
        dropped.append(st["area_dropped"])
    assert dropped[0] > 0
    assert all(b < a for a, b in zip(dropped, dropped[1:]))
