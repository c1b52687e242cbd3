"""Adjoint FMM (lens_deflect_adjoint) against the oracle's FP64 gradient,
central finite differences of the GPU forward, and the full differentiable
light-curve chain (reduced differentiation workload)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import autograd, lens, synth

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def reduced_c5(n=1000, seed=0):
    f = synth.config_uniform(seed=seed, n=n, kappa_star=0.3, kappa_s=0.2, gamma=0.4,
                             mass_range=(0.5, 1.5))
    return f


def rel_norm(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("leaf", [4, 16])
def test_adjoint_matches_oracle_gradient(leaf):
    f = reduced_c5()
    L = 6.0
    rays = synth.random_rays(3, 20000, (-L, -L), (L, L))
    gy = np.random.default_rng(4).normal(size=rays.shape)
    with lens.LensFMM(T(f.stars), T(f.masses), f.kappa_s, f.gamma, p=48, leaf_size=leaf,
                      prec=lens.FP64, target_box=(-L, L, -L, L)) as P:
        gxy, gm, gkg = P.adjoint(T(rays), T(gy))
    rgxy, rgm, rgkg = oracle.adjoint(f.stars, f.masses, rays, gy)
    e1, e2 = rel_norm(gxy.cpu().numpy(), rgxy), rel_norm(gm.cpu().numpy(), rgm)
    print("adjoint rel err: positions %.2e masses %.2e" % (e1, e2))
    assert e1 < 1e-10 and e2 < 1e-10
    np.testing.assert_allclose(gkg.cpu().numpy(), rgkg, rtol=1e-12)


def test_adjoint_on_clustered_tree():
    rng = np.random.default_rng(0)
    centres = rng.uniform(-5, 5, (12, 2))
    stars = (centres[:, None, :] + rng.normal(0, 0.2, (12, 60, 2))).reshape(-1, 2)
    m = rng.uniform(0.5, 1.5, len(stars))
    rays = synth.random_rays(1, 8000, (-6, -6), (6, 6))
    gy = rng.normal(size=rays.shape)
    with lens.LensFMM(T(stars), T(m), 0.1, 0.2, p=48, leaf_size=4, prec=lens.FP64,
                      target_box=(-6, 6, -6, 6)) as P:
        info = P.info()
        gxy, gm, _ = P.adjoint(T(rays), T(gy))
    assert info["n_w"] > 0 and info["n_x"] > 0
    rgxy, rgm, _ = oracle.adjoint(stars, m, rays, gy)
    assert rel_norm(gxy.cpu().numpy(), rgxy) < 1e-10
    assert rel_norm(gm.cpu().numpy(), rgm) < 1e-10


@pytest.mark.parametrize("prec", [lens.FP64, lens.FP32_BULK])
def test_recomputed_tree_gives_the_same_gradient(prec):
    # backward with the tree rebuilt (the large-N* mode) = backward on the
    # forward pass's tree; both match the oracle's float64 gradient
    f = reduced_c5(n=700, seed=3)
    L = 4.0
    rays = T(synth.random_rays(9, 5000, (-L, -L), (L, L)))
    W = np.random.default_rng(10).normal(size=(5000, 2))
    grads = []
    for rec in (False, True):
        stars = T(f.stars).requires_grad_(True)
        masses = T(f.masses).requires_grad_(True)
        y = autograd.deflect(stars, masses, f.kappa_s, f.gamma, rays, p=40, leaf_size=8, prec=prec,
                             target_box=(-L, L, -L, L), recompute=rec)
        (y * T(W)).sum().backward()
        grads.append((stars.grad.cpu().numpy(), masses.grad.cpu().numpy()))
    # rays reach their leaves' tiles in any order (an atomic cursor), so the
    # sums regroup: ~1e-16 in float64, float32 partial sums by up to ~1e-7
    same = 1e-12 if prec == lens.FP64 else 1e-6
    assert rel_norm(grads[1][0], grads[0][0]) < same
    assert rel_norm(grads[1][1], grads[0][1]) < same
    rgxy, rgm, _ = oracle.adjoint(f.stars, f.masses, rays.cpu().numpy(), W)
    tol = 1e-9 if prec == lens.FP64 else FP32_GRAD_TOL
    assert rel_norm(grads[1][0], rgxy) < tol
    assert rel_norm(grads[1][1], rgm) < tol


# float32-bulk plans run the adjoint's per-ray and per-pair operators (P2P^T,
# L2P^T, M2P^T) in float32 -- float-float offsets, compensated sums -- and its
# transposed translations in float64: the gradient is held to the float32
# form's 2e-5, normwise (each pair term carries ~1e-7 relative error).
FP32_GRAD_TOL = 2e-5


@pytest.mark.parametrize("clustered", [False, True])
def test_float32_bulk_adjoint_matches_oracle_gradient(clustered):
    rng = np.random.default_rng(11)
    if clustered:
        centres = rng.uniform(-5, 5, (12, 2))
        stars = (centres[:, None, :] + rng.normal(0, 0.2, (12, 60, 2))).reshape(-1, 2)
        m = rng.uniform(0.5, 1.5, len(stars))
        ks, g, leaf = 0.1, 0.2, 4
    else:
        f = reduced_c5(n=2000, seed=5)
        stars, m, ks, g, leaf = f.stars, f.masses, f.kappa_s, f.gamma, 16
    L = 6.0
    rays = synth.random_rays(12, 20000, (-L, -L), (L, L))
    # rays exactly on two stars and 1e-4 ER from a third (stars in the box)
    inside = np.nonzero((np.abs(stars[:, 0]) < L - 1) & (np.abs(stars[:, 1]) < L - 1))[0][:3]
    rays[:3] = stars[inside]
    rays[2] += 1e-4
    gy = rng.normal(size=rays.shape)
    with lens.LensFMM(T(stars), T(m), ks, g, p=24, leaf_size=leaf, prec=lens.FP32_BULK,
                      target_box=(-L, L, -L, L)) as P:
        info = P.info()
        gxy, gm, gkg = P.adjoint(T(rays), T(gy))
    if clustered:
        assert info["n_w"] > 0 and info["n_x"] > 0
    rgxy, rgm, rgkg = oracle.adjoint(stars, m, rays, gy)
    e1, e2 = rel_norm(gxy.cpu().numpy(), rgxy), rel_norm(gm.cpu().numpy(), rgm)
    print("float32-bulk adjoint rel err: positions %.2e masses %.2e" % (e1, e2))
    assert e1 < FP32_GRAD_TOL and e2 < FP32_GRAD_TOL
    np.testing.assert_allclose(gkg.cpu().numpy(), rgkg, rtol=1e-12)


def test_autograd_matches_central_differences():
    f = reduced_c5(n=400, seed=2)
    L = 4.0
    rays = T(synth.random_rays(5, 3000, (-L, -L), (L, L)))
    W = T(np.random.default_rng(6).normal(size=(3000, 2)))
    stars = T(f.stars).requires_grad_(True)
    masses = T(f.masses).requires_grad_(True)
    ks = torch.tensor(f.kappa_s, dtype=torch.float64, device="cuda", requires_grad=True)
    g = torch.tensor(f.gamma, dtype=torch.float64, device="cuda", requires_grad=True)
    box = (-L, L, -L, L)

    def loss(st, ms, k_, g_):
        return (autograd.deflect(st, ms, k_, g_, rays, p=48, leaf_size=8, target_box=box) * W).sum()

    Lv = loss(stars, masses, ks, g)
    Lv.backward()
    h = 1e-5
    rng = np.random.default_rng(7)
    with torch.no_grad():
        for j in rng.choice(f.n, 16, replace=False):
            for c in range(2):
                sp = stars.detach().clone(); sp[j, c] += h
                sm = stars.detach().clone(); sm[j, c] -= h
                fd = (loss(sp, masses.detach(), ks.detach(), g.detach()) -
                      loss(sm, masses.detach(), ks.detach(), g.detach())).item() / (2 * h)
                assert stars.grad[j, c].item() == pytest.approx(fd, rel=1e-6, abs=1e-7)
            mp = masses.detach().clone(); mp[j] += h
            mm = masses.detach().clone(); mm[j] -= h
            fd = (loss(stars.detach(), mp, ks.detach(), g.detach()) -
                  loss(stars.detach(), mm, ks.detach(), g.detach())).item() / (2 * h)
            assert masses.grad[j].item() == pytest.approx(fd, rel=1e-6, abs=1e-7)
        for var, grad in ((0, ks.grad), (1, g.grad)):
            kp = [ks.detach().item(), g.detach().item()]
            km = list(kp)
            kp[var] += h
            km[var] -= h
            fd = (loss(stars.detach(), masses.detach(), kp[0], kp[1]) -
                  loss(stars.detach(), masses.detach(), km[0], km[1])).item() / (2 * h)
            assert grad.item() == pytest.approx(fd, rel=1e-6)


def test_light_curve_chain_matches_oracle():
    # reduced differentiation workload: loss = sum_k (F_k - T_k)^2 of a
    # Gaussian-source light curve along a track; target from a perturbed field
    f = reduced_c5(n=1000, seed=0)
    ft = synth.perturbed(f, seed=1, sd=0.01)
    grid = synth.Grid(x0=-6.0, y0=-2.5, h=0.02, nx=600, ny=250)
    rays = grid.corners().reshape(-1, 2)
    s = synth.light_curve_track(256, length=1.0)
    sig, w = 0.05, grid.h ** 2
    box = (-6.0, 6.0, -2.5, 2.5)
    with torch.no_grad():
        yt = autograd.deflect(T(ft.stars), T(ft.masses), ft.kappa_s, ft.gamma, T(rays), p=40,
                              leaf_size=8, target_box=box)
        Tk = lens.light_curve(yt, w, T(s), sig)
    stars = T(f.stars).requires_grad_(True)
    masses = T(f.masses).requires_grad_(True)
    y = autograd.deflect(stars, masses, f.kappa_s, f.gamma, T(rays), p=40, leaf_size=8,
                         target_box=box)
    F = autograd.light_curve(y, w, T(s), sig)
    loss = ((F - Tk) ** 2).sum()
    loss.backward()
    # oracle chain
    y_o = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, rays)
    F_o = oracle.light_curve(y_o, w, s, sig)
    np.testing.assert_allclose(F.detach().cpu().numpy(), F_o, rtol=1e-8, atol=1e-10)
    gy_o = oracle.light_curve_grad(y_o, w, s, sig, F_o, Tk.cpu().numpy())
    gxy_o, gm_o, _ = oracle.adjoint(f.stars, f.masses, rays, gy_o)
    assert rel_norm(stars.grad.cpu().numpy(), gxy_o) < 1e-8
    assert rel_norm(masses.grad.cpu().numpy(), gm_o) < 1e-8
