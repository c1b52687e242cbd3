"""Parity at the full sizes of the other workload configurations:

* clustered primordial-black-hole field (1e6 lenses in 1e3 Plummer clusters,
  log-normal masses, leaf 64, 4096^2 map over 100 ER);
* extreme magnification near a critical curve (2e5 stars, mu ~ 286,
  8192^2 map over 2 ER, ~2.2e10 cells in chunks);
* elliptical NFW halo of 1e7 particles, deflection only on a 4096^2 grid;
* the differentiation workload (1e5 stars, 3e6 rays, 2048-sample Gaussian
  light curve): adjoint gradients against central differences.

Deflections are checked on sampled rays against the oracle's direct sum,
maps on full-width bands against the oracle's IPM of the same deflections,
whole maps through their ledgers and mean magnification."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import autograd, dist as ldist, lens, synth
from helpers import alpha_rel_err

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def grid_box(g):
    return (g.x0, g.x0 + g.nx * g.h, g.y0, g.y0 + g.ny * g.h)


def ledger_ok(st, rel=1e-6):
    led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
    return abs(led - st["area_total"]) <= rel * st["area_total"]


def band_check(f, P, row0, nrows, cap=64):
    band = ldist.strip_grid(f.grid, row0, nrows)
    y = P.deflect_grid(band).cpu().numpy()
    ref, st_ref = oracle.ipm_map(y, band.h, f.box, f.npx, f.npy, bbox_cap=cap)
    mp, st = P.ipm_map(band, f.box, f.npx, f.npy, bbox_cap=cap)
    mp = mp.cpu().numpy()
    good = np.abs(ref) > 1e-3 * np.abs(ref).max()
    e = np.mean(np.abs(mp[good] - ref[good]) / np.abs(ref[good]))
    assert e < 1e-3, e
    assert st["cells_dropped"] == pytest.approx(st_ref["cells_dropped"], rel=1e-3, abs=5)
    # total flux to 1e-6, up to the cells the two sides drop differently at
    # the cap (each moves at most one cell area h^2)
    slack = 1e-6 * st_ref["area_total"] + abs(st["cells_dropped"] - st_ref["cells_dropped"]) * band.h ** 2
    for k in ("area_in_map", "area_outside"):
        assert abs(st[k] - st_ref[k]) <= slack, (k, st[k], st_ref[k], slack)
    return e, int(good.sum())


@pytest.fixture(scope="module")
def c3():
    return synth.c3_clustered(seed=0)


def test_clustered_field_deflections(c3):
    f = c3
    idx, x = synth.subsample_grid_rays(11, f.grid, 2048)
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=16, leaf_size=64,
                      prec=lens.FP32_BULK, target_box=grid_box(f.grid)) as P:
        y32 = P.deflect(T(x)).cpu().numpy()
        info = P.info()
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=48, leaf_size=64,
                      prec=lens.FP64, target_box=grid_box(f.grid)) as P:
        y64 = P.deflect(T(x[:512])).cpu().numpy()
    e32 = alpha_rel_err(y32, y_ref, x, f.kappa_s, f.gamma)
    e64 = alpha_rel_err(y64, y_ref[:512], x[:512], f.kappa_s, f.gamma)
    print("C3: levels %d, FP32-bulk max %.2e, FP64 max %.2e" % (info["levels"], e32.max(), e64.max()))
    assert info["n_w"] > 0 and info["n_x"] > 0  # the adaptive lists are exercised
    assert e32.max() < 2e-5
    assert e64.max() < 1e-10


def test_clustered_field_map(c3):
    f = c3
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=16, leaf_size=64,
                      prec=lens.FP32_BULK, target_box=grid_box(f.grid)) as P:
        e, n = band_check(f, P, f.grid.ny // 2 - 40, 80)
        mp, st = P.ipm_map(f.grid, f.box, f.npx, f.npy, bbox_cap=64)
    print("C3 band map: mean rel err %.2e over %d pixels" % (e, n))
    assert ledger_ok(st)
    assert abs(mp.sum().item() * (100.0 / 4096) ** 2 - st["area_in_map"]) <= 1e-6 * st["area_total"]
    assert st["rays"] >= (f.grid.nx + 1) * (f.grid.ny + 1)


@pytest.fixture(scope="module")
def c4():
    return synth.c4_critical(seed=0)


def test_critical_curve_deflections_and_band(c4):
    f = c4
    idx, x = synth.subsample_grid_rays(12, f.grid, 2048)
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    # the configuration bench.py times (leaf 4, p 16)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=16, leaf_size=4,
                      prec=lens.FP32_BULK, target_box=grid_box(f.grid)) as P:
        y = P.deflect(T(x)).cpu().numpy()
        e = alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma)
        print("C4 sampled: max %.2e" % e.max())
        assert e.max() < 2e-5
        eb, n = band_check(f, P, f.grid.ny // 2, 4)
        print("C4 band map (4 x %d cells): mean rel err %.2e over %d pixels" % (f.grid.nx, eb, n))


def test_critical_curve_full_map(c4):
    # ~2.2e10 cells, split into chunks by free device memory
    f = c4
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=16, leaf_size=4,
                      prec=lens.FP32_BULK, target_box=grid_box(f.grid)) as P:
        mp, st = P.ipm_map(f.grid, f.box, f.npx, f.npy, bbox_cap=64)
    assert st["chunks"] >= 2
    assert ledger_ok(st)
    assert abs(mp.sum().item() * (2.0 / 8192) ** 2 - st["area_in_map"]) <= 1e-6 * st["area_total"]
    mu = 1.0 / abs((1 - 0.82) ** 2 - 0.17 ** 2)
    print("C4: %d chunks, %.3g cells, interior mean magnification %.2f (macro %.2f)"
          % (st["chunks"], st["cells"], mp[512:-512, 512:-512].mean().item(), mu))


def test_critical_curve_mean_magnification(c4):
    # The workload's shooting region (3% margin) misses rays that stars
    # deflect into the map: in the direction compressed by |1-k-g| = 0.01 a
    # source-plane deflection of ~0.3 ER is ~30 ER in the image plane.  With
    # margins of ~3 |alpha|_rms / |1 -+ k - g| on both axes (and coarser cells,
    # 0.06 per unlensed pixel) the interior mean returns to the macro value.
    f = c4
    h = 1e-3
    g = synth.shooting_grid(0.82, 0.17, 1.0, h, margin_frac=1.0, margin_min=3.0)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=16, leaf_size=8,
                      prec=lens.FP32_BULK, target_box=grid_box(g)) as P:
        mp, st = P.ipm_map(g, f.box, 2048, 2048, bbox_cap=64)
    assert ledger_ok(st)
    mu = 1.0 / abs((1 - 0.82) ** 2 - 0.17 ** 2)
    inner = mp[128:-128, 128:-128].mean().item()
    print("C4 wide margins: %.3g cells, interior mean magnification %.2f (macro %.2f)"
          % (st["cells"], inner, mu))
    assert abs(inner / mu - 1) < 0.05


def test_nfw_halo_deflections():
    f = synth.nfw_halo(seed=0)
    g = f.grid
    idx, x = synth.subsample_grid_rays(13, g, 384)
    y_ref = oracle.deflect(f.stars, f.masses, 0.0, 0.0, x)
    # the configuration bench.py times (leaf 128, p 12)
    with lens.LensFMM(T(f.stars), T(f.masses), 0.0, 0.0, p=12, leaf_size=128,
                      prec=lens.FP32_BULK, target_box=grid_box(g)) as P:
        yg = P.deflect_grid(g)
        y = yg.cpu().numpy()[idx[:, 1], idx[:, 0]]
        info = P.info()
    e = alpha_rel_err(y, y_ref, x, 0.0, 0.0)
    print("NFW 1e7 particles: %d levels, grid max err %.2e" % (info["levels"], e.max()))
    assert yg.shape[:2] == (g.ny + 1, g.nx + 1)
    assert e.max() < 2e-5


def test_differentiation_workload_gradients():
    # full differentiation workload: 1e5 stars, 6000 x 500 cells of rays,
    # 2048-sample Gaussian light curve (sigma 0.05 ER) against the curve of a
    # perturbed field; gradients by the adjoint FMM vs central differences
    f = synth.c5_differentiable(seed=0)
    g = f.grid
    rays = T(g.corners().reshape(-1, 2))
    s = T(synth.light_curve_track(2048, length=5.0))
    sig, w = 0.05, g.h ** 2
    box = grid_box(g)
    ft = synth.perturbed(f, seed=1, sd=0.01)
    with torch.no_grad():
        yt = autograd.deflect(T(ft.stars), T(ft.masses), ft.kappa_s, ft.gamma, rays, p=32,
                              leaf_size=16, target_box=box)
        Tk = lens.light_curve(yt, w, s, sig)

    # the float64 form at p 32; the float32-bulk form at p 24, as bench.py times it
    def loss(st, ms, k_, g_, prec=lens.FP64):
        y = autograd.deflect(st, ms, k_, g_, rays, p=32 if prec == lens.FP64 else 24, leaf_size=16,
                             prec=prec, target_box=box)
        return ((autograd.light_curve(y, w, s, sig) - Tk) ** 2).sum()

    stars = T(f.stars).requires_grad_(True)
    masses = T(f.masses).requires_grad_(True)
    ks = torch.tensor(f.kappa_s, dtype=torch.float64, device="cuda", requires_grad=True)
    gm = torch.tensor(f.gamma, dtype=torch.float64, device="cuda", requires_grad=True)
    L0 = loss(stars, masses, ks, gm)
    L0.backward()
    assert L0.item() > 0
    # the float32-bulk forward with the same float64 adjoint
    st32 = T(f.stars).requires_grad_(True)
    loss(st32, T(f.masses), f.kappa_s, f.gamma, prec=lens.FP32_BULK).backward()
    inside = np.nonzero((np.abs(f.stars[:, 0]) < 28) & (np.abs(f.stars[:, 1]) < 2.3))[0]
    gs = stars.grad.cpu().numpy()
    assert np.linalg.norm(st32.grad.cpu().numpy()[inside] - gs[inside]) <= 1e-3 * np.linalg.norm(gs[inside])
    # central differences at h and 2h combined by Richardson extrapolation,
    # (4 D(h) - D(2h)) / 3, which cancels the O(h^2) term: a change of kappa_s
    # or gamma moves every ray by h |x| (|x| up to 30 ER) against a source of
    # 0.05 ER, where the plain central difference is off by ~(h x / sigma)^2 / 6
    h = 1e-5

    def richardson(ev):
        d1 = (ev(h) - ev(-h)) / (2 * h)
        d2 = (ev(2 * h) - ev(-2 * h)) / (4 * h)
        return (4 * d1 - d2) / 3

    def check(name, g_adj, fd):
        rel = abs(g_adj - fd) / max(abs(fd), 1e-300)
        print("C5 %s: adjoint %.12g central %.12g rel %.2e" % (name, g_adj, fd, rel))
        assert g_adj == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(gs).max())

    rng = np.random.default_rng(3)
    with torch.no_grad():
        M0 = masses.detach()
        for j in rng.choice(inside, 4, replace=False):
            for c in range(2):
                def ev(d, j=j, c=c):
                    sp = stars.detach().clone()
                    sp[j, c] += d
                    return loss(sp, M0, f.kappa_s, f.gamma).item()
                check("dL/dx[%d,%d]" % (j, c), gs[j, c], richardson(ev))

            def evm(d, j=j):
                mp = M0.clone()
                mp[j] += d
                return loss(stars.detach(), mp, f.kappa_s, f.gamma).item()
            check("dL/dm[%d]" % j, masses.grad[j].item(), richardson(evm))
        for var, grad in ((0, ks.grad), (1, gm.grad)):
            def evk(d, var=var):
                kg = [f.kappa_s, f.gamma]
                kg[var] += d
                return loss(stars.detach(), M0, kg[0], kg[1]).item()
            check("dL/d%s" % ("kappa_s", "gamma")[var], grad.item(), richardson(evk))
