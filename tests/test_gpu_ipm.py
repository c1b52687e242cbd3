"""FMM-IPM map (lens_ipm_map) against the oracle's scalar IPM applied to the
oracle's own deflections, plus exact and ledger invariants."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens, synth

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def ledger_ok(st, rel=1e-6):
    led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
    return abs(led - st["area_total"]) <= rel * st["area_total"]


def map_rel_err(mp, ref):
    """mean per-pixel relative error over pixels with signal"""
    good = np.abs(ref) > 1e-3 * np.abs(ref).max()
    return np.mean(np.abs(mp[good] - ref[good]) / np.abs(ref[good]))


@pytest.fixture(scope="module")
def c1_oracle():
    f = synth.c1_plain(seed=0)
    g = f.grid
    y = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, g.corners().reshape(-1, 2))
    y = y.reshape(g.ny + 1, g.nx + 1, 2)
    mp, st = oracle.ipm_map(y, g.h, f.box, f.npx, f.npy)
    return f, mp, st


@pytest.mark.parametrize("prec,p", [(lens.FP64, 40), (lens.FP32_BULK, 24)])
def test_c1_map_matches_oracle(c1_oracle, prec, p):
    f, ref, st_ref = c1_oracle
    g = f.grid
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=p, leaf_size=16, prec=prec,
                      target_box=(-10, 10, -10, 10)) as P:
        mp, st = P.ipm_map(g, f.box, f.npx, f.npy)
        mp2, st2 = P.ipm_map(g, f.box, f.npx, f.npy, max_cells_per_chunk=7 * g.nx + 3)
    mp, mp2 = mp.cpu().numpy(), mp2.cpu().numpy()
    e = map_rel_err(mp, ref)
    print("C1 map mean rel err", e, "chunks", st2["chunks"])
    assert e < 1e-3
    assert ledger_ok(st) and ledger_ok(st2)
    assert abs(st["area_in_map"] - st_ref["area_in_map"]) <= 1e-6 * st_ref["area_total"]
    assert abs(np.sum(mp) * 0.01 - st["area_in_map"]) <= 1e-6 * st["area_total"]
    assert st2["chunks"] > 50
    # float32 accumulation in a different order: equal to ~1e-6
    np.testing.assert_allclose(mp2, mp, rtol=2e-6, atol=1e-6 * np.abs(mp).max())


def test_affine_lens_map_is_inverse_determinant():
    # a single massless lens: y = diag(1-ks-g, 1-ks+g) x exactly
    ks, g = 0.25, 0.3
    grid = synth.Grid(x0=-6.0, y0=-6.0, h=0.021, nx=571, ny=571)
    with lens.LensFMM(T([[0.0, 0.0]]), T([0.0]), ks, g, p=4, leaf_size=4, prec=lens.FP32_BULK,
                      target_box=(-6, 6, -6, 6)) as P:
        mp, st = P.ipm_map(grid, (-1.0, 1.0, -2.0, 2.0), 64, 80)
    det = (1 - ks - g) * (1 - ks + g)
    np.testing.assert_allclose(mp.cpu().numpy(), 1 / abs(det), rtol=2e-6)
    assert ledger_ok(st)


def test_flushed_map_of_an_expanding_affine_lens():
    # kappa_s = -3, gamma = 0 and no stars: y = 4 x, so every cell maps to a
    # square 4 h = 0.084 on a side, 8.4 pixels of 0.01 (the large-cell path:
    # row bands, crossed pixels and the difference array), and every pixel
    # of the window is covered with magnification 1/16.  A 40 x 40 map
    # flushes its float32 accumulators into the float-float running map every
    # 64 x 1600 cells, three times over the 571^2 grid, in chunks of 20 rows.
    ks, g = -3.0, 0.0
    grid = synth.Grid(x0=-6.0, y0=-6.0, h=0.021, nx=571, ny=571)
    with lens.LensFMM(T([[0.0, 0.0]]), T([0.0]), ks, g, p=4, leaf_size=4, prec=lens.FP32_BULK,
                      target_box=(-6, 6, -6, 6)) as P:
        mp, st = P.ipm_map(grid, (-0.2, 0.2, -0.2, 0.2), 40, 40, max_cells_per_chunk=20 * 571)
    assert st["chunks"] == 29
    np.testing.assert_allclose(mp.cpu().numpy(), 1 / 16, rtol=2e-6)
    assert ledger_ok(st)


def test_point_lens_magnification():
    box = (-2.0, 2.0, -2.0, 2.0)
    h = 0.0125
    grid = synth.Grid(x0=-3.5 + 0.5 * h, y0=-3.5 + 0.5 * h, h=h, nx=560, ny=560)
    with lens.LensFMM(T([[0.0, 0.0]]), T([1.0]), 0.0, 0.0, p=16, leaf_size=4,
                      prec=lens.FP32_BULK, target_box=(-3.6, 3.6, -3.6, 3.6)) as P:
        mp, st = P.ipm_map(grid, box, 40, 40, bbox_cap=64)
    mp = mp.cpu().numpy()
    c = -2.0 + (np.arange(40) + 0.5) * 0.1
    U, V = np.meshgrid(c, c)
    r = np.hypot(U, V)
    mu = (r * r + 2) / (r * np.sqrt(r * r + 4))
    far = r >= 0.5
    assert np.mean(np.abs(mp[far] - mu[far]) / mu[far]) < 5e-3
    assert ledger_ok(st)


def test_cap_drops_and_ledger_agree_with_oracle():
    f = synth.config_uniform(seed=4, n=600, kappa_star=0.4, kappa_s=0.0, gamma=0.1)
    grid = synth.Grid(x0=-4.0, y0=-4.0, h=0.02, nx=400, ny=400)
    y = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, grid.corners().reshape(-1, 2))
    y = y.reshape(grid.ny + 1, grid.nx + 1, 2)
    box = (-2.0, 2.0, -2.0, 2.0)
    ref, st_ref = oracle.ipm_map(y, grid.h, box, 200, 200, bbox_cap=3)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=40, leaf_size=8,
                      prec=lens.FP64, target_box=(-4, 4, -4, 4)) as P:
        mp, st = P.ipm_map(grid, box, 200, 200, bbox_cap=3)
    assert st["cells_dropped"] == st_ref["cells_dropped"] > 0
    assert st["area_dropped"] == pytest.approx(st_ref["area_dropped"], rel=1e-12)
    assert ledger_ok(st)
    assert map_rel_err(mp.cpu().numpy(), ref) < 1e-3
