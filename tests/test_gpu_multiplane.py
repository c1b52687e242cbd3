"""Rays through several lens planes (lens_multiplane_deflect,
lens_multiplane_ipm_map) against the oracle's multi-plane recursion (Sec. 1:
ray tracing through several lens planes, the mapping repeated plane by
plane).

float64 plans (p = 48): positions on every plane and y end to end within
1e-10 of the oracle.  float32-bulk plans (p = 24): each plane's step against
the oracle's Eq. 1 at the positions the GPU sent the rays to (2e-5), since
near a star on a later plane an upstream float32 error is magnified by the
lens map's Jacobian (~1/d^2) whatever the kernels do.  Maps: the oracle's
IPM of the oracle's multi-plane deflections, mean per-pixel error 1e-3 and a
closed ledger."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00354_gb300 import lens, synth

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def planes3():
    rng = np.random.default_rng(21)
    out = []
    for n, r, ks, g in ((2000, 12.0, 0.05, 0.1), (1500, 10.0, 0.0, -0.05), (1000, 9.0, 0.1, 0.02)):
        out.append((synth.uniform_disk(rng, n, r), rng.uniform(0.2, 1.0, n), ks, g))
    beta = np.array([[0.0, 0.45, 0.7], [0.0, 0.0, 0.5], [0.0, 0.0, 0.0]])
    return out, beta


def rel(y, y_ref, x):
    """|dy| / max(|x - y_ref|, 1e-3 rms(x - y_ref)): the total deflection's scale."""
    al = x - y_ref
    mag = np.hypot(al[:, 0], al[:, 1])
    return np.hypot(*(y - y_ref).T) / np.maximum(mag, 1e-3 * np.sqrt(np.mean(mag ** 2)))


def gpu_planes(planes):
    return [(T(s), T(m), ks, g) for s, m, ks, g in planes]


def test_fp64_matches_oracle_end_to_end():
    planes, beta = planes3()
    x = synth.random_rays(22, 3000, (-6, -4), (6, 4))
    y, xp = lens.multiplane_deflect(gpu_planes(planes), beta, T(x), p=48, leaf_size=16,
                                    prec=lens.FP64, planes_out=True)
    y_ref, xp_ref = oracle.multiplane_deflect(planes, beta, x, planes_out=True)
    assert rel(y.cpu().numpy(), y_ref, x).max() < 1e-10
    for i in range(1, 3):
        assert rel(xp[i].cpu().numpy(), xp_ref[i], x).max() < 1e-10
    np.testing.assert_array_equal(xp[0].cpu().numpy(), x)


def test_fp32_bulk_each_plane_matches_eq1():
    planes, beta = planes3()
    x = synth.random_rays(23, 3000, (-6, -4), (6, 4))
    y, xp = lens.multiplane_deflect(gpu_planes(planes), beta, T(x), p=24, leaf_size=16,
                                    prec=lens.FP32_BULK, planes_out=True)
    y, xp = y.cpu().numpy(), xp.cpu().numpy()
    # each plane's deflection as the GPU applied it, recovered from the
    # positions it sent the rays to (x_j = x - sum_{i<j} beta_ij alpha_i,
    # y = x - sum_i alpha_i), against the oracle's Eq. 1 at the same points
    K = len(planes)
    got = []
    for j in range(1, K + 1):
        w = [beta[i, j] if j < K else 1.0 for i in range(j)]
        rest = sum(w[i] * got[i] for i in range(j - 1)) if j > 1 else 0.0
        pos = xp[j] if j < K else y
        got.append((x - pos - rest) / w[j - 1])
    for i, (st, ms, ks, g) in enumerate(planes):
        _, a = oracle.deflect(st, ms, 0.0, 0.0, xp[i], alpha=True)
        a = a + np.array([ks + g, ks - g]) * xp[i]
        mag = np.hypot(a[:, 0], a[:, 1])
        e = np.hypot(*(got[i] - a).T) / np.maximum(mag, 1e-3 * np.sqrt(np.mean(mag ** 2)))
        assert e.max() < 2e-5, (i, e.max())


def test_empty_middle_plane_and_arguments():
    planes, beta = planes3()
    x = synth.random_rays(24, 1000, (-5, -3), (5, 3))
    empty = (np.zeros((0, 2)), np.zeros(0), 0.0, 0.0)
    y3 = lens.multiplane_deflect(gpu_planes([planes[0], empty, planes[2]]), beta, T(x), p=40,
                                 leaf_size=16, prec=lens.FP64).cpu().numpy()
    y2_ref = oracle.multiplane_deflect([planes[0], planes[2]],
                                       np.array([[0.0, beta[0, 2]], [0.0, 0.0]]), x)
    assert rel(y3, y2_ref, x).max() < 1e-10
    with pytest.raises(lens.LensError) as e:
        lens.multiplane_deflect([], np.zeros((0, 0)), T(x))
    assert e.value.status == lens.LENS_EINVAL
    bad = beta.copy()
    bad[0, 1] = np.nan
    with pytest.raises(lens.LensError) as e:
        lens.multiplane_deflect(gpu_planes(planes), bad, T(x))
    assert e.value.status == lens.LENS_EINVAL
    xn = x.copy()
    xn[5, 1] = np.inf
    with pytest.raises(lens.LensError) as e:
        lens.multiplane_deflect(gpu_planes(planes), beta, T(xn))
    assert e.value.status == lens.LENS_EDOMAIN
    # no rays: nothing to do
    assert lens.multiplane_deflect(gpu_planes(planes), beta, T(np.zeros((0, 2)))).shape == (0, 2)


@pytest.mark.parametrize("prec,p", [(lens.FP64, 32), (lens.FP32_BULK, 24)])
def test_two_plane_map_matches_oracle(prec, p):
    f = synth.c1_plain(seed=0)
    rng = np.random.default_rng(25)
    second = (synth.uniform_disk(rng, 600, 30.0), rng.uniform(0.3, 1.0, 600), 0.1, 0.05)
    planes = [(f.stars, f.masses, f.kappa_s, f.gamma), second]
    beta = np.array([[0.0, 0.6], [0.0, 0.0]])
    g = f.grid
    mp, st = lens.multiplane_ipm_map(gpu_planes(planes), beta, g, f.box, f.npx, f.npy, p=p,
                                     leaf_size=16, prec=prec, max_cells_per_chunk=90_000)
    assert st["chunks"] > 1
    y_ref = oracle.multiplane_deflect(planes, beta, g.corners().reshape(-1, 2))
    mp_ref, st_ref = oracle.ipm_map(y_ref.reshape(g.ny + 1, g.nx + 1, 2), g.h, f.box, f.npx, f.npy)
    mp = mp.cpu().numpy()
    good = np.abs(mp_ref) > 1e-3 * np.abs(mp_ref).max()  # pixels with signal
    assert np.mean(np.abs(mp[good] - mp_ref[good]) / np.abs(mp_ref[good])) < 1e-3
    led = st["area_in_map"] + st["area_outside"] + st["area_dropped"] + st["area_degenerate"]
    assert abs(led - st["area_total"]) <= 1e-6 * st["area_total"]
    assert abs(st["area_in_map"] - st_ref["area_in_map"]) <= 1e-6 * st_ref["area_total"]
