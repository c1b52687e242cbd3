"""The fused deflection + IPM kernel (lens_ipm_map_ex with LENS_MAP_FUSED;
Sec. 2.4 steps 3-4 with no corner array in device memory) against the
oracle's IPM of the oracle's deflections (mean per-pixel error 1e-3, ledger
closed to 1e-6), and against the separate-kernel path, which must give the
same map up to the order of the float32 additions: every cell's polygon is
formed from the same corner bits on both paths."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import dist as ldist, lens, synth

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def ledger_ok(st, rel=1e-6):
    led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
    return abs(led - st["area_total"]) <= rel * st["area_total"]


def map_rel_err(mp, ref):
    good = np.abs(ref) > 1e-3 * np.abs(ref).max()
    return np.mean(np.abs(mp[good] - ref[good]) / np.abs(ref[good]))


def same_maps(a, b, sa, sb):
    np.testing.assert_allclose(a, b, rtol=2e-6, atol=1e-6 * np.abs(b).max())
    for k in ("cells_dropped", "cells_degenerate", "cells_queued", "cells_ext"):
        assert sa[k] == sb[k], k
    for k in ("area_in_map", "area_outside", "area_dropped"):
        assert abs(sa[k] - sb[k]) <= 1e-6 * sb["area_total"], k
    assert sa["ipm_updates"] == sb["ipm_updates"]
    # corner rays count each chunk seam twice
    if sa["chunks"] == sb["chunks"]:
        assert sa["rays"] == sb["rays"]


@pytest.fixture(scope="module")
def c1_oracle():
    f = synth.c1_plain(seed=0)
    g = f.grid
    y = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, g.corners().reshape(-1, 2))
    mp, st = oracle.ipm_map(y.reshape(g.ny + 1, g.nx + 1, 2), g.h, f.box, f.npx, f.npy)
    return f, mp, st


@pytest.mark.parametrize("masses", ["equal", "varied"])
def test_fused_map_matches_oracle_and_separate_path(c1_oracle, masses):
    f, ref, st_ref = c1_oracle
    g = f.grid
    m = f.masses if masses == "equal" else np.random.default_rng(5).uniform(0.5, 1.5, f.n)
    if masses == "varied":
        y = oracle.deflect(f.stars, m, f.kappa_s, f.gamma, g.corners().reshape(-1, 2))
        ref, st_ref = oracle.ipm_map(y.reshape(g.ny + 1, g.nx + 1, 2), g.h, f.box, f.npx, f.npy)
    with lens.LensFMM(T(f.stars), T(m), f.kappa_s, f.gamma, p=24, leaf_size=16,
                      prec=lens.FP32_BULK, target_box=(-10, 10, -10, 10)) as P:
        mf, sf = P.ipm_map(g, f.box, f.npx, f.npy, fused=True)
        ms, ss = P.ipm_map(g, f.box, f.npx, f.npy, fused=False)
        mc, sc = P.ipm_map(g, f.box, f.npx, f.npy, fused=True, max_cells_per_chunk=7 * g.nx + 3)
    assert sf["fused"] == 1 and ss["fused"] == 0 and sc["chunks"] > 30
    mf, ms, mc = mf.cpu().numpy(), ms.cpu().numpy(), mc.cpu().numpy()
    assert map_rel_err(mf, ref) < 1e-3
    assert ledger_ok(sf) and ledger_ok(sc)
    assert abs(sf["area_in_map"] - st_ref["area_in_map"]) <= 1e-6 * st_ref["area_total"]
    same_maps(mf, ms, sf, ss)
    np.testing.assert_allclose(mc, mf, rtol=2e-6, atol=1e-6 * np.abs(mf).max())
    # the overlapping work items evaluate a few corners twice, no fewer
    assert sf["rays_evaluated"] >= sf["rays"]


def test_fused_with_leaves_wider_than_a_work_item():
    # few stars over a fine grid: leaves of ~700 x 700 rays, split into
    # several column segments and many row bands; cells near the stars are
    # ill-conditioned and large
    f = synth.config_uniform(seed=8, n=60, kappa_star=0.3, kappa_s=0.1, gamma=0.2)
    g = synth.Grid(x0=-6.0, y0=-6.0, h=0.01, nx=1200, ny=1200)
    box = (-4.0, 4.0, -4.0, 4.0)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=24, leaf_size=8,
                      prec=lens.FP32_BULK, target_box=(-6, 6, -6, 6)) as P:
        mf, sf = P.ipm_map(g, box, 160, 160, bbox_cap=64, fused=True)
        ms, ss = P.ipm_map(g, box, 160, 160, bbox_cap=64, fused=False)
        y = P.deflect_grid(g).cpu().numpy()
    ref, st_ref = oracle.ipm_map(y, g.h, box, 160, 160, bbox_cap=64)
    mf, ms = mf.cpu().numpy(), ms.cpu().numpy()
    assert sf["cells_ext"] > 0 and sf["cells_queued"] > 0
    assert ledger_ok(sf)
    same_maps(mf, ms, sf, ss)
    assert map_rel_err(mf, ref) < 1e-3
    assert sf["cells_dropped"] == pytest.approx(st_ref["cells_dropped"], abs=2)


def test_fused_clustered_band_and_refinement():
    # adaptive tree (leaves from ~0.1 to ~100 ER), U/V/W/X lists, a band of
    # the clustered workload's grid; then critical-cell refinement on top
    f = synth.c3_clustered(seed=0, n_clusters=40, per_cluster=200)
    band = ldist.strip_grid(f.grid, f.grid.ny // 2 - 30, 60)
    tb = (band.x0, band.x0 + band.nx * band.h, band.y0, band.y0 + band.ny * band.h)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=16, leaf_size=16,
                      prec=lens.FP32_BULK, target_box=tb) as P:
        y = P.deflect_grid(band).cpu().numpy()
        mf, sf = P.ipm_map(band, f.box, 512, 512, bbox_cap=64, fused=True)
        ms, ss = P.ipm_map(band, f.box, 512, 512, bbox_cap=64, fused=False)
        rf, srf = P.ipm_map(band, f.box, 512, 512, bbox_cap=16, refine_levels=2, fused=True)
        rs, srs = P.ipm_map(band, f.box, 512, 512, bbox_cap=16, refine_levels=2, fused=False)
    ref, _ = oracle.ipm_map(y, band.h, f.box, 512, 512, bbox_cap=64)
    mf, ms = mf.cpu().numpy(), ms.cpu().numpy()
    assert map_rel_err(mf, ref) < 1e-3
    assert ledger_ok(sf)
    same_maps(mf, ms, sf, ss)
    assert srf["cells_refined"] == srs["cells_refined"] > 0
    np.testing.assert_allclose(rf.cpu().numpy(), rs.cpu().numpy(), rtol=2e-6,
                               atol=1e-6 * np.abs(rs.cpu().numpy()).max())


def test_fused_needs_a_float32_bulk_plan():
    f = synth.config_uniform(seed=9, n=100, kappa_star=0.3, kappa_s=0.0, gamma=0.0)
    g = synth.Grid(x0=-2.0, y0=-2.0, h=0.05, nx=80, ny=80)
    with lens.LensFMM(T(f.stars), T(f.masses), 0.0, 0.0, p=16, leaf_size=8, prec=lens.FP64,
                      target_box=(-2, 2, -2, 2)) as P:
        with pytest.raises(lens.LensError) as e:
            P.ipm_map(g, (-1, 1, -1, 1), 20, 20, fused=True)
        assert e.value.status == lens.LENS_EINVAL
        _, st = P.ipm_map(g, (-1, 1, -1, 1), 20, 20)
        assert st["fused"] == 0
