"""Critical-cell refinement (lens_ipm_map_refined) against the oracle's
refined IPM: cells whose pixel box exceeds the cap are split 2 x 2, the new
corner rays deflected through the plan, instead of dropped."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens, synth

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def maps(stars, masses, ks, g, grid, box, npx, npy, cap, levels, prec=lens.FP64, p=40, leaf=8):
    y = oracle.deflect(stars, masses, ks, g, grid.corners().reshape(-1, 2))
    y = y.reshape(grid.ny + 1, grid.nx + 1, 2)
    ref, st_ref = oracle.ipm_map_refined(y, grid.x0, grid.y0, grid.h, stars, masses, ks, g, box,
                                         npx, npy, cap, levels)
    target = (grid.x0, grid.x0 + grid.nx * grid.h, grid.y0, grid.y0 + grid.ny * grid.h)
    with lens.LensFMM(T(stars), T(masses), ks, g, p=p, leaf_size=leaf, prec=prec,
                      target_box=target) as P:
        mp, st = P.ipm_map(grid, box, npx, npy, bbox_cap=cap, refine_levels=levels)
    return mp.cpu().numpy(), st, ref, st_ref


def rel_err(mp, ref):
    good = np.abs(ref) > 1e-3 * np.abs(ref).max()
    return np.mean(np.abs(mp[good] - ref[good]) / np.abs(ref[good]))


def ledger_ok(st, rel=1e-6):
    led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
    return abs(led - st["area_total"]) <= rel * st["area_total"]


def test_affine_lens_refined_equals_uncapped():
    star, m = np.array([[0.3, -0.2]]), np.array([0.0])
    ks, g = -2.0, 0.5
    grid = synth.Grid(x0=-0.5, y0=-0.4, h=0.1, nx=10, ny=8)
    box = (-1.5, 1.5, -1.5, 1.5)
    mp, st, ref, st_ref = maps(star, m, ks, g, grid, box, 30, 30, 4, 3)
    assert st["cells_refined"] > 0 and st["cells_dropped"] == 0
    np.testing.assert_allclose(mp, ref, rtol=2e-5, atol=1e-6 * np.abs(ref).max())
    assert ledger_ok(st)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_point_lens_refinement_matches_oracle(levels):
    box = (-2.0, 2.0, -2.0, 2.0)
    h = 0.05
    grid = synth.Grid(x0=-2.0 + 0.5 * h, y0=-2.0 + 0.3 * h, h=h, nx=80, ny=80)
    star, m = np.zeros((1, 2)), np.array([1.0])
    mp, st, ref, st_ref = maps(star, m, 0.0, 0.0, grid, box, 40, 40, 8, levels, p=24, leaf=4)
    assert st["cells_refined"] > 0
    assert rel_err(mp, ref) < 1e-3
    assert ledger_ok(st)
    for k in ("area_in_map", "area_outside", "area_dropped"):
        assert st[k] == pytest.approx(st_ref[k], rel=1e-4, abs=1e-6 * st_ref["area_total"])


@pytest.mark.parametrize("prec,p", [(lens.FP64, 40), (lens.FP32_BULK, 24)])
def test_star_field_refinement_matches_oracle(prec, p):
    f = synth.config_uniform(seed=6, n=400, kappa_star=0.4, kappa_s=0.05, gamma=0.15)
    grid = synth.Grid(x0=-3.0, y0=-3.0, h=0.04, nx=150, ny=150)
    box = (-2.0, 2.0, -2.0, 2.0)
    mp, st, ref, st_ref = maps(f.stars, f.masses, f.kappa_s, f.gamma, grid, box, 100, 100, 3, 2,
                               prec=prec, p=p)
    assert st["cells_refined"] > 0
    assert rel_err(mp, ref) < 1e-3
    assert ledger_ok(st)
    assert st["area_dropped"] == pytest.approx(st_ref["area_dropped"], rel=1e-3,
                                               abs=1e-6 * st_ref["area_total"])
    # refinement books less area as dropped than the plain cap
    _, st0, _, _ = maps(f.stars, f.masses, f.kappa_s, f.gamma, grid, box, 100, 100, 3, 0,
                        prec=prec, p=p)
    assert st["area_dropped"] < st0["area_dropped"]
