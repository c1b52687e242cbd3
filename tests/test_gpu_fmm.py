"""FMM deflection (lens_fmm_build + lens_deflect / lens_deflect_grid) against
the FP64 oracle: error falls geometrically with p, meets 1e-10 (FP64 form) and
2e-5 (FP32-bulk form), on uniform and clustered (adaptive) fields, full grids
with ragged leaf tiles, Jacobians, and the error paths."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens, synth
from helpers import alpha_rel_err

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def plan_for(f, p, leaf, prec, box=None):
    return lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=p, leaf_size=leaf,
                        prec=prec, target_box=box)


@pytest.fixture(scope="module")
def c1():
    f = synth.c1_plain(seed=0)
    x = synth.random_rays(7, 4000, (-10, -10), (10, 10))
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    return f, x, y_ref


def test_error_falls_geometrically_with_p(c1):
    f, x, y_ref = c1
    errs = []
    for p in (4, 8, 12, 16, 24, 32):
        with plan_for(f, p, 16, lens.FP64, (-10, 10, -10, 10)) as P:
            y = P.deflect(T(x)).cpu().numpy()
        errs.append(alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma).max())
    print("max rel err vs p:", dict(zip((4, 8, 12, 16, 24, 32), errs)))
    for a, b in zip(errs, errs[1:]):
        assert b < 0.6 * a
    # p = 12 (the plain-method configuration): 0.55^13 a-priori ratio
    assert errs[2] < 1e-3


@pytest.mark.parametrize("prec,p,tol", [(lens.FP64, 48, 1e-10), (lens.FP32_BULK, 24, 2e-5)])
def test_stated_tolerances(c1, prec, p, tol):
    f, x, y_ref = c1
    with plan_for(f, p, 16, prec, (-10, 10, -10, 10)) as P:
        y = P.deflect(T(x)).cpu().numpy()
    err = alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma)
    print("prec", prec, "p", p, "max", err.max(), "p99.9", np.quantile(err, 0.999))
    assert err.max() < tol


def test_full_grid_matches_oracle_and_ray_path():
    # every corner of a grid that spans many leaves, with a ragged last tile
    f = synth.config_uniform(seed=9, n=3000, kappa_star=0.4, kappa_s=0.05, gamma=0.3,
                             radius=15.0)
    grid = synth.Grid(x0=-6.0, y0=-5.0, h=0.037, nx=301, ny=257)
    xc = grid.corners().reshape(-1, 2)
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, xc)
    with plan_for(f, 40, 8, lens.FP64, (-6.0, 6.0, -5.0, 5.0)) as P:
        yg = P.deflect_grid(grid).cpu().numpy().reshape(-1, 2)
        yr = P.deflect(T(xc)).cpu().numpy()
        band = P.deflect_grid(grid, row0=100, nrows=33).cpu().numpy()
        info = P.info()
    assert info["n_active_leaves"] > 50
    assert alpha_rel_err(yg, y_ref, xc, f.kappa_s, f.gamma).max() < 1e-10
    assert alpha_rel_err(yr, y_ref, xc, f.kappa_s, f.gamma).max() < 1e-10
    np.testing.assert_array_equal(band, yg.reshape(grid.ny + 1, grid.nx + 1, 2)[100:133])


def test_full_grid_fp32_bulk_matches_oracle():
    # the float32-bulk grid path (the map path's kernel, y output) at every
    # corner of a grid spanning many leaves, ragged tiles included
    f = synth.config_uniform(seed=9, n=3000, kappa_star=0.4, kappa_s=0.05, gamma=0.3,
                             radius=15.0)
    grid = synth.Grid(x0=-6.0, y0=-5.0, h=0.037, nx=301, ny=257)
    xc = grid.corners().reshape(-1, 2)
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, xc)
    for leaf in (4, 8, 16):
        with plan_for(f, 24, leaf, lens.FP32_BULK, (-6.0, 6.0, -5.0, 5.0)) as P:
            yg = P.deflect_grid(grid).cpu().numpy().reshape(-1, 2)
            yr = P.deflect(T(xc)).cpu().numpy()
            bands = [P.deflect_grid(grid, row0=r0, nrows=n).cpu().numpy()
                     for r0, n in ((0, 1), (7, 8), (100, 33), (250, 8))]
        eg = alpha_rel_err(yg, y_ref, xc, f.kappa_s, f.gamma)
        er = alpha_rel_err(yr, y_ref, xc, f.kappa_s, f.gamma)
        print("leaf %d: grid %.2e ray %.2e" % (leaf, eg.max(), er.max()))
        assert eg.max() < 2e-5 and er.max() < 2e-5, leaf
        # a band of rows evaluates its corners like the whole grid: the
        # near field's grid-unit origin of a leaf does not move with the
        # band, so only the float-float rounding of the leaf-centre offset
        # (~1e-14 ER) may differ
        full = yg.reshape(grid.ny + 1, grid.nx + 1, 2)
        for (r0, n), b in zip(((0, 1), (7, 8), (100, 33), (250, 8)), bands):
            assert np.abs(b - full[r0:r0 + n]).max() < 1e-12, (leaf, r0)


def clustered(seed=0, nc=30, per=80):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-8, 8, (nc, 2))
    u = rng.random((nc, per)) * (400.0 / 401.0)
    r = 0.3 * np.sqrt(u / (1 - u))
    t = rng.uniform(0, 2 * np.pi, (nc, per))
    stars = (centres[:, None, :] + np.stack([r * np.cos(t), r * np.sin(t)], -1)).reshape(-1, 2)
    m = rng.lognormal(0, 1, nc * per)
    return synth.Field(stars=stars, masses=m, kappa_s=0.3, gamma=0.3, kappa_star=0.2)


def test_adaptive_tree_on_clustered_field():
    # deep, unbalanced tree: U, V, W and X lists all populated
    f = clustered()
    x = np.concatenate([synth.random_rays(1, 2000, (-9, -9), (9, 9)),
                        f.stars[::7] + 1e-3])  # rays inside the clusters too
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    with plan_for(f, 48, 4, lens.FP64, (-9.5, 9.5, -9.5, 9.5)) as P:
        y = P.deflect(T(x)).cpu().numpy()
        info = P.info()
    print(info)
    assert info["n_w"] > 0 and info["n_x"] > 0 and info["levels"] > 8
    err = alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma)
    assert err.max() < 1e-10, err.max()
    with plan_for(f, 24, 16, lens.FP32_BULK, (-9.5, 9.5, -9.5, 9.5)) as P:
        y32 = P.deflect(T(x)).cpu().numpy()
    assert alpha_rel_err(y32, y_ref, x, f.kappa_s, f.gamma).max() < 2e-5


def test_tree_deeper_than_the_partial_sort():
    # 1000 field stars over ~60 ER plus 1000 stars within 1e-5 ER: ~26 levels,
    # far below the levels the build sorts first for 2000 stars, so the keys
    # are sorted again in full and the splits recounted
    rng = np.random.default_rng(5)
    wide = synth.uniform_disk(rng, 1000, 30.0)
    tight = synth.uniform_disk(rng, 1000, 1e-5, center=(1.25, -0.75))
    f = synth.Field(stars=np.concatenate([wide, tight]), masses=rng.uniform(0.5, 1.5, 2000),
                    kappa_s=0.1, gamma=0.2, kappa_star=0.0)
    x = np.concatenate([synth.random_rays(6, 1500, (-20, -20), (20, 20)),
                        tight[::5] + 3e-6, np.array([[1.25, -0.75], [1.25 + 1e-4, -0.75]])])
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    with plan_for(f, 48, 8, lens.FP64, (-20.5, 20.5, -20.5, 20.5)) as P:
        y = P.deflect(T(x)).cpu().numpy()
        info = P.info()
    assert info["levels"] > 20
    assert alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma).max() < 1e-10
    with plan_for(f, 24, 8, lens.FP32_BULK, (-20.5, 20.5, -20.5, 20.5)) as P:
        y32 = P.deflect(T(x)).cpu().numpy()
    assert alpha_rel_err(y32, y_ref, x, f.kappa_s, f.gamma).max() < 2e-5


@pytest.mark.parametrize("m0", [1.0, 0.5, 0.37])
def test_equal_mass_fields(m0):
    # equal masses: the float32 near field sums unweighted and scales once
    # (1 and 0.5 are exact in float32; 0.37 is not and takes the general path)
    f = synth.config_uniform(seed=9, n=3000, kappa_star=0.4, kappa_s=0.1, gamma=0.2)
    f.masses = np.full(f.n, m0)
    x = np.concatenate([synth.random_rays(10, 3000, (-8, -8), (8, 8)), f.stars[:200] + 1e-4])
    x = x[np.all(np.abs(x) < 8, axis=1)]
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    with plan_for(f, 24, 8, lens.FP32_BULK, (-8.5, 8.5, -8.5, 8.5)) as P:
        y = P.deflect(T(x)).cpu().numpy()
    assert alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma).max() < 2e-5


@pytest.mark.parametrize("prec,tol", [(lens.FP64, 1e-8), (lens.FP32_BULK, 2e-4)])
def test_jacobian(prec, tol):
    f = synth.config_uniform(seed=1, n=800, kappa_star=0.3, kappa_s=0.2, gamma=0.4)
    x = synth.random_rays(2, 1500, (-5, -5), (5, 5))
    _, jac_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x, jacobian=True)
    with plan_for(f, 40, 8, prec, (-5, 5, -5, 5)) as P:
        _, jac = P.deflect(T(x), jacobian=True)
    d = np.abs(jac.cpu().numpy() - jac_ref).reshape(-1, 4).max(1)
    sc = np.maximum(np.abs(jac_ref).reshape(-1, 4).max(1), 1.0)
    assert (d / sc).max() < tol


@pytest.mark.parametrize("prec,tol", [(lens.FP64, 1e-10), (lens.FP32_BULK, 2e-5)])
def test_rays_exactly_on_stars(prec, tol):
    # a star exactly at a ray contributes nothing (the oracle skips r == 0);
    # with and without the Jacobian, through the near field of every leaf
    f = synth.config_uniform(seed=4, n=600, kappa_star=0.3, kappa_s=0.1, gamma=0.2)
    inside = np.all(np.abs(f.stars) < 4.0, axis=1)
    x = np.concatenate([f.stars[inside][:200], synth.random_rays(8, 100, (-4, -4), (4, 4))])
    y_ref, jac_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x, jacobian=True)
    with plan_for(f, 40, 8, prec, (-4, 4, -4, 4)) as P:
        y = P.deflect(T(x)).cpu().numpy()
        yj, jac = P.deflect(T(x), jacobian=True)
    assert np.all(np.isfinite(y)) and np.all(np.isfinite(jac.cpu().numpy()))
    assert alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma).max() < tol
    assert alpha_rel_err(yj.cpu().numpy(), y_ref, x, f.kappa_s, f.gamma).max() < tol
    d = np.abs(jac.cpu().numpy() - jac_ref).reshape(-1, 4).max(1)
    sc = np.maximum(np.abs(jac_ref).reshape(-1, 4).max(1), 1.0)
    assert (d / sc).max() < (1e-8 if prec == lens.FP64 else 2e-4)


def test_evaluation_on_another_stream_waits_for_the_build():
    # the expansions finish on the plan's own stream after the build returns;
    # calls on any stream wait for them (and the adjoint for the tree)
    f = synth.config_uniform(seed=5, n=20000, kappa_star=0.4, kappa_s=0.1, gamma=0.2)
    x = synth.random_rays(6, 50000, (-20, -20), (20, 20))
    box = (-20, 20, -20, 20)
    xs = T(x)
    gy = T(np.random.default_rng(2).normal(size=x.shape))
    ref = {}
    for prec in (lens.FP32_BULK, lens.FP64):
        with plan_for(f, 24, 8, prec, box) as P:
            ref[prec] = (P.deflect(xs).cpu().numpy(), P.adjoint(xs, gy)[0].cpu().numpy())
        s2 = torch.cuda.Stream()
        with plan_for(f, 24, 8, prec, box) as P:
            with torch.cuda.stream(s2):
                y2 = P.deflect(xs, stream=s2)
                g2 = P.adjoint(xs, gy, stream=s2)[0]
            s2.synchronize()
            np.testing.assert_array_equal(y2.cpu().numpy(), ref[prec][0])
            # the adjoint's sums regroup with the order rays reach their leaves
            # (an atomic cursor): ~1e-16 in float64, ~1e-7 in float32 partials
            tol = 1e-12 if prec == lens.FP64 else 1e-5
            g2n, gr = g2.cpu().numpy(), ref[prec][1]
            assert np.linalg.norm(g2n - gr) <= tol * np.linalg.norm(gr)
            assert P.info()["ms_build"] > 0


def test_plans_on_the_torch_allocator_match_the_default_pool():
    # the build allocates on three streams (the caller's, and the plan's two
    # for the upward pass and the lists); through torch's caching allocator
    # the plan must give the same bits as with the library's own pool
    f = synth.config_uniform(seed=7, n=30000, kappa_star=0.45, kappa_s=0.0, gamma=0.45)
    g = synth.Grid(x0=-15.0, y0=-15.0, h=0.05, nx=600, ny=600)
    box = (g.x0, g.x0 + g.nx * g.h, g.y0, g.y0 + g.ny * g.h)
    x = T(synth.random_rays(8, 40000, (-15, -15), (15, 15)))
    out = []
    for torch_alloc in (False, True):
        with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=16, leaf_size=8,
                          prec=lens.FP32_BULK, target_box=box, use_torch_allocator=torch_alloc) as P:
            y = P.deflect(x)
            mp, st = P.ipm_map(g, (-4.0, 4.0, -4.0, 4.0), 200, 200)
            out.append((y.cpu().numpy(), mp.cpu().numpy(), st["area_in_map"]))
    np.testing.assert_array_equal(out[1][0], out[0][0])
    # the map's float32 atomics add in a schedule-dependent order
    np.testing.assert_allclose(out[1][1], out[0][1], rtol=1e-5, atol=1e-6 * np.abs(out[0][1]).max())
    assert abs(out[1][2] - out[0][2]) <= 1e-6 * abs(out[0][2])


def test_tiny_fields():
    for n, leaf in ((1, 16), (5, 16), (40, 1), (17, 16)):
        f = synth.config_uniform(seed=n, n=n, kappa_star=0.3, kappa_s=0.0, gamma=0.1)
        L = max(1.0, np.abs(f.stars).max())
        x = synth.random_rays(5, 300, (-L, -L), (L, L))
        y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
        with plan_for(f, 40, leaf, lens.FP64, (-L, L, -L, L)) as P:
            y = P.deflect(T(x)).cpu().numpy()
        assert alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma).max() < 1e-10, (n, leaf)


def test_no_target_box_means_whole_root():
    f = synth.config_uniform(seed=3, n=500, kappa_star=0.3, kappa_s=0.0, gamma=0.1)
    lo, hi = f.stars.min(0), f.stars.max(0)
    x = synth.random_rays(6, 500, lo, hi)
    y_ref = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    with plan_for(f, 40, 8, lens.FP64, None) as P:
        y = P.deflect(T(x)).cpu().numpy()
        assert P.info()["n_active_boxes"] == P.info()["n_boxes"]
    assert alpha_rel_err(y, y_ref, x, f.kappa_s, f.gamma).max() < 1e-10


def test_error_paths():
    f = synth.config_uniform(seed=0, n=100, kappa_star=0.3, kappa_s=0, gamma=0)
    with plan_for(f, 8, 8, lens.FP32_BULK, (-1, 1, -1, 1)) as P:
        with pytest.raises(lens.LensError) as e:
            P.deflect(T([[0.0, 0.0], [1e6, 5.0]]))   # second ray outside the root
        assert e.value.status == lens.LENS_EDOMAIN
        with pytest.raises(lens.LensError) as e:
            P.deflect(T([[float("nan"), 0.0]]))
        assert e.value.status == lens.LENS_EDOMAIN
        with pytest.raises(lens.LensError) as e:
            P.deflect_grid(synth.Grid(-2, -2, 0.1, 40, 40))
        assert e.value.status == lens.LENS_EDOMAIN
        assert P.deflect(T(np.zeros((0, 2)))).shape == (0, 2)
    # coincident stars beyond leaf_size: depth cap
    stars = np.zeros((20, 2))
    with pytest.raises(lens.LensError) as e:
        lens.LensFMM(T(stars), T(np.ones(20)), p=8, leaf_size=4)
    assert e.value.status == lens.LENS_EDEPTH
    with pytest.raises(lens.LensError) as e:
        lens.LensFMM(T(np.full((4, 2), np.nan)), T(np.ones(4)), p=8, leaf_size=4)
    assert e.value.status == lens.LENS_EINVAL
