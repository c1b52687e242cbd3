"""lens_direct_deflect_noalloc: the direct sum for callers that may not
allocate device memory (a host application that owns the device-memory
budget, a service with a capped pool); its scratch is one static device
array.  Checked through the C ABI on two calls in a row with different
inputs: bit for bit against lens_direct_deflect in its float32 form (the
same kernel on the same operands, so the same roundings) and against the
oracle's Eq. 1 within the float32 tolerance 2e-5; plus the size limit.
Collected last on purpose; passes alone in a fresh process as well as after
the others."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
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
        # the allocating entry point runs the same kernel on the same split
        # stars: identical bits
        assert torch.equal(y, y_ref)
        assert torch.equal(jac, jac_ref)
        # and the definition itself (Eq. 1 by the oracle's float64 direct sum)
        yo, jo = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x, jacobian=True)
        err = alpha_rel_err(y.cpu().numpy(), yo, x, f.kappa_s, f.gamma)
        assert err.max() < 2e-5
        dj = np.abs(jac.cpu().numpy() - jo).max()
        assert dj <= 1e-4 * np.abs(jo).max()


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
