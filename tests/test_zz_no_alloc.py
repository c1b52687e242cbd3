"""lens_direct_deflect_noalloc: the direct sum for callers that may not
allocate device memory (the library uses a fixed static scratch array).
Checked against lens_direct_deflect (float32 form) through the C ABI on two
calls in a row with different inputs, plus the size limit.  Collected last
on purpose; passes alone in a fresh process as well as after the others."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2211_00354_gb300 import lens, synth
from helpers import alpha_rel_err

pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def call_noalloc(lib, stars, masses, ks, g, rays, y, jac):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.lens_direct_deflect_noalloc(stars.data_ptr(), masses.data_ptr(), stars.shape[0],
                                           ks, g, rays.data_ptr(), rays.shape[0], y.data_ptr(),
                                           jac.data_ptr() if jac is not None else None, stream)


def test_noalloc_matches_direct_on_two_calls_in_a_row():
    lib = lens.load()
    cases = [(synth.config_uniform(seed=11, n=20000, kappa_star=0.4, kappa_s=0.1, gamma=0.3),
              synth.random_rays(12, 4099, (-20, -20), (20, 20))),
             (synth.config_uniform(seed=13, n=777, kappa_star=0.2, kappa_s=0.0, gamma=0.0),
              synth.random_rays(14, 1500, (-8, -8), (8, 8)))]
    for f, x in cases:
        stars, masses, rays = T(f.stars), T(f.masses), T(x)
        y = torch.full_like(rays, float("nan"))
        jac = torch.full((rays.shape[0], 2, 2), float("nan"), dtype=torch.float64, device="cuda")
        st = call_noalloc(lib, stars, masses, f.kappa_s, f.gamma, rays, y, jac)
        assert st == lens.LENS_OK, lib.lens_last_error()
        y_ref, jac_ref = lens.direct_deflect(stars, masses, f.kappa_s, f.gamma, rays,
                                             prec=lens.FP32_BULK, jacobian=True)
        torch.cuda.synchronize()
        err = alpha_rel_err(y.cpu().numpy(), y_ref.cpu().numpy(), x, f.kappa_s, f.gamma)
        assert err.max() < 2e-5
        dj = np.abs(jac.cpu().numpy() - jac_ref.cpu().numpy()).max()
        assert dj <= 1e-4 * np.abs(jac_ref.cpu().numpy()).max()


def test_noalloc_rejects_more_stars_than_its_scratch():
    lib = lens.load()
    n = lens.NOALLOC_MAX_STARS + 1
    stars = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    masses = torch.ones(n, dtype=torch.float64, device="cuda")
    rays = torch.ones((4, 2), dtype=torch.float64, device="cuda")
    y = torch.empty_like(rays)
    st = call_noalloc(lib, stars, masses, 0.0, 0.0, rays, y, None)
    assert st == lens.LENS_EINVAL
    assert b"262144" in lib.lens_last_error()
