"""Edge cases of the map path against the oracle's scalar IPM: a grid that
lands wholly outside the map, a one-pixel map, a one-cell grid, and a lens
that collapses every cell to a segment (all cells degenerate)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens, synth

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_and_oracle_maps(f, grid, box, npx, npy, cap=0, p=40, prec=lens.FP64):
    y = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, grid.corners().reshape(-1, 2))
    y = y.reshape(grid.ny + 1, grid.nx + 1, 2)
    ref, st_ref = oracle.ipm_map(y, grid.h, box, npx, npy, bbox_cap=cap)
    target = (grid.x0, grid.x0 + grid.nx * grid.h, grid.y0, grid.y0 + grid.ny * grid.h)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=p, leaf_size=8, prec=prec,
                      target_box=target) as P:
        mp, st = P.ipm_map(grid, box, npx, npy, bbox_cap=cap)
    return mp.cpu().numpy(), st, ref, st_ref


def field(seed=0, n=300):
    return synth.config_uniform(seed=seed, n=n, kappa_star=0.3, kappa_s=0.1, gamma=0.2)


def test_grid_wholly_outside_the_map():
    f = field()
    grid = synth.Grid(x0=-4.0, y0=-4.0, h=0.05, nx=160, ny=160)
    box = (50.0, 60.0, 50.0, 60.0)  # far from every deflected corner
    mp, st, ref, st_ref = gpu_and_oracle_maps(f, grid, box, 32, 32)
    assert np.all(mp == 0) and np.all(ref == 0)
    assert st["area_in_map"] == 0.0
    assert st["area_outside"] == pytest.approx(st["area_total"], rel=1e-6)
    assert st["area_outside"] == pytest.approx(st_ref["area_outside"], rel=1e-6)


@pytest.mark.parametrize("prec", [lens.FP64, lens.FP32_BULK])
def test_one_pixel_map(prec):
    f = field(seed=1)
    grid = synth.Grid(x0=-3.0, y0=-3.0, h=0.04, nx=150, ny=150)
    box = (-1.0, 1.0, -1.0, 1.0)
    mp, st, ref, st_ref = gpu_and_oracle_maps(f, grid, box, 1, 1, prec=prec, p=40 if prec == lens.FP64 else 24)
    assert mp.shape == (1, 1)
    assert mp[0, 0] == pytest.approx(ref[0, 0], rel=1e-4)
    # 22500 cells on one pixel: the float32 accumulators are flushed every
    # 64 cells per pixel (one grid row of 150 cells here), so the map and the
    # float32 ledger agree to ~150 float32 roundings
    assert st["chunks"] == grid.ny
    assert mp[0, 0] * 4.0 == pytest.approx(st["area_in_map"], rel=2e-5)
    assert st["area_in_map"] == pytest.approx(st_ref["area_in_map"], rel=1e-4)


def test_one_cell_grid():
    f = field(seed=2, n=50)
    grid = synth.Grid(x0=0.3, y0=-0.2, h=0.5, nx=1, ny=1)
    box = (-2.0, 2.0, -2.0, 2.0)
    mp, st, ref, st_ref = gpu_and_oracle_maps(f, grid, box, 40, 40)
    assert st["cells"] == 1
    # the clipping runs in float32 for well-conditioned cells: per-pixel
    # agreement to float32 rounding of the pixel-unit corner positions
    assert np.count_nonzero(ref) > 4
    np.testing.assert_allclose(mp, ref, rtol=1e-4, atol=1e-5 * np.abs(ref).max())
    for k in ("area_in_map", "area_outside", "area_dropped", "area_degenerate"):
        # the ledger sums float32 fractions: 1 - sum(fractions) leaves ~2^-24
        assert st[k] == pytest.approx(st_ref[k], rel=1e-5, abs=1e-6 * st_ref["area_total"])


def test_every_cell_degenerate():
    # a = 1 - kappa_s - gamma = 0 and a massless star: y1 = 0 for every ray,
    # every cell has zero area and is booked as degenerate, nothing is mapped
    f = synth.Field(stars=np.array([[0.5, 0.5]]), masses=np.array([0.0]), kappa_s=0.6,
                    gamma=0.4, kappa_star=0.0)
    grid = synth.Grid(x0=-1.0, y0=-1.0, h=0.05, nx=40, ny=40)
    box = (-1.0, 1.0, -1.0, 1.0)
    mp, st, ref, st_ref = gpu_and_oracle_maps(f, grid, box, 20, 20)
    assert np.all(mp == 0) and np.all(ref == 0)
    assert st["cells_degenerate"] == st_ref["cells_degenerate"] == grid.nx * grid.ny
    assert st["area_degenerate"] == pytest.approx(st["area_total"], rel=1e-9)


def test_cells_spanning_the_whole_map_without_a_cap():
    # a point lens inside a coarse grid: the cells next to the lens map to
    # polygons hundreds of pixels across (rows of a large cell wider than the
    # per-warp staging), no cap, so every one is apportioned
    f = synth.Field(stars=np.array([[0.013, -0.021]]), masses=np.array([1.0]), kappa_s=0.0,
                    gamma=0.0, kappa_star=0.0)
    grid = synth.Grid(x0=-1.5, y0=-1.5, h=0.05, nx=60, ny=60)
    box = (-3.0, 3.0, -3.0, 3.0)
    npx = npy = 300
    mp, st, ref, st_ref = gpu_and_oracle_maps(f, grid, box, npx, npy, cap=0)
    # the widest polygon's pixel box, from the oracle's deflections
    y = oracle.deflect(f.stars, f.masses, 0.0, 0.0, grid.corners().reshape(-1, 2))
    y = y.reshape(grid.ny + 1, grid.nx + 1, 2)
    u = (y[..., 0] - box[0]) / 0.02
    wmax = max(np.ptp(u[j:j + 2, i:i + 2]) for j in range(grid.ny) for i in range(grid.nx))
    assert wmax > 200
    good = np.abs(ref) > 1e-3 * np.abs(ref).max()
    assert np.mean(np.abs(mp[good] - ref[good]) / np.abs(ref[good])) < 1e-3
    for k in ("area_in_map", "area_outside"):
        assert st[k] == pytest.approx(st_ref[k], rel=1e-5, abs=1e-6 * st_ref["area_total"])
    assert st["cells_dropped"] == 0
