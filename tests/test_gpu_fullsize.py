"""The high-magnification map workload at full size, in the configuration
bench.py times (N* = 1.5e6, 32699 x 3493 cells, 2000^2 map, FP32-bulk p=16,
leaf 8, bbox cap 64): sampled deflections vs the oracle, grid path vs ray
path, the IPM on a full-width band of rows vs the oracle's IPM of the same
deflections, and whole-map invariants (flux ledger, mean magnification)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import dist as ldist
from paper_2211_00354_gb300 import lens, synth
from helpers import alpha_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    f = synth.c2_high_mag(seed=0)
    g = f.grid
    target = (g.x0, g.x0 + g.nx * g.h, g.y0, g.y0 + g.ny * g.h)
    dev = torch.device("cuda")
    P = lens.LensFMM(torch.tensor(f.stars, device=dev), torch.tensor(f.masses, device=dev),
                     f.kappa_s, f.gamma, p=16, leaf_size=8, prec=lens.FP32_BULK,
                     target_box=target)
    yield f, P
    P.close()


def test_sampled_rays_match_oracle(c2):
    f, P = c2
    idx, x = synth.subsample_grid_rays(21, f.grid, 2048)
    y = P.deflect(torch.tensor(x, device="cuda")).cpu().numpy()
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    err = alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma)
    print("C2 sampled: max %.2e p99.9 %.2e" % (err.max(), np.quantile(err, 0.999)))
    assert err.max() < 2e-5


def test_grid_path_matches_ray_path_on_a_band(c2):
    f, P = c2
    g = f.grid
    yb = P.deflect_grid(g, row0=1700, nrows=3).cpu().numpy().reshape(-1, 2)
    xc = g.corners()[1700:1703].reshape(-1, 2)
    yr = P.deflect(torch.tensor(xc, device="cuda")).cpu().numpy()
    assert alpha_rel_err(yb, yr, xc, f.kappa_s, f.gamma).max() < 2e-5
    sel = np.random.default_rng(3).choice(len(xc), 500, replace=False)
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, xc[sel])
    assert alpha_rel_err(yb[sel], y_ref, xc[sel], f.kappa_s, f.gamma).max() < 2e-5


def test_ipm_on_a_full_width_band_matches_oracle(c2):
    f, P = c2
    band = ldist.strip_grid(f.grid, 1650, 120)   # 120 x 32699 cells through the middle
    y = P.deflect_grid(band).cpu().numpy()
    ref, st_ref = oracle.ipm_map(y, band.h, f.box, f.npx, f.npy, bbox_cap=64)
    mp, st = P.ipm_map(band, f.box, f.npx, f.npy, bbox_cap=64)
    mp = mp.cpu().numpy()
    good = np.abs(ref) > 1e-3 * np.abs(ref).max()
    e = np.mean(np.abs(mp[good] - ref[good]) / np.abs(ref[good]))
    print("C2 band map: mean rel err %.2e over %d pixels" % (e, good.sum()))
    assert e < 1e-3
    assert st["cells_dropped"] == pytest.approx(st_ref["cells_dropped"], rel=1e-3, abs=5)
    # total flux to 1e-6, up to the cells the two sides drop differently
    # (float32 against float64 pixel coordinates at the 64-pixel cap): each
    # moves at most one cell area h^2 between the ledger's categories
    slack = 1e-6 * st_ref["area_total"] + abs(st["cells_dropped"] - st_ref["cells_dropped"]) * band.h ** 2
    for k in ("area_in_map", "area_outside"):
        print("C2 band %s: %.9g vs %.9g (slack %.3g)" % (k, st[k], st_ref[k], slack))
        assert abs(st[k] - st_ref[k]) <= slack


def test_full_map_invariants(c2):
    f, P = c2
    mp, st = P.ipm_map(f.grid, f.box, f.npx, f.npy, bbox_cap=64)
    led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
    assert abs(led - st["area_total"]) <= 1e-6 * st["area_total"]
    assert st["rays"] == (f.grid.nx + 1) * (f.grid.ny + 1) + (st["chunks"] - 1) * (f.grid.nx + 1)
    inner = mp[100:-100, 100:-100].mean().item()
    print("C2 mean interior magnification %.4f (macro 10)" % inner)
    assert abs(inner / 10.0 - 1) < 0.05
