"""Lensing potential by direct sum -- TEST INFRASTRUCTURE ONLY, float64 numpy.

psi(x) = sum_i m_i ln|x - x_i| + kappa_s |x|^2 / 2 + gamma (x1^2 - x2^2) / 2:
the potential whose gradient is x - y for the lens equation of Eq. 1 with
its smooth field (the potential of the cosmological-lens example of
Sec. 2.5).  A star exactly at a ray contributes nothing.  Rays in chunks,
each chunk's sum over stars by numpy's pairwise summation.
"""
from __future__ import annotations

import numpy as np


def potential(stars, masses, kappa_s, gamma, rays, chunk=256):
    stars = np.asarray(stars, dtype=np.float64).reshape(-1, 2)
    masses = np.asarray(masses, dtype=np.float64).reshape(-1)
    rays = np.asarray(rays, dtype=np.float64).reshape(-1, 2)
    out = np.empty(rays.shape[0])
    for r0 in range(0, rays.shape[0], chunk):
        x = rays[r0:r0 + chunk]
        d2 = (x[:, None, 0] - stars[None, :, 0]) ** 2 + (x[:, None, 1] - stars[None, :, 1]) ** 2
        with np.errstate(divide="ignore"):
            lg = np.where(d2 > 0.0, 0.5 * np.log(np.where(d2 > 0.0, d2, 1.0)), 0.0)
        out[r0:r0 + chunk] = np.sum(lg * masses[None, :], axis=1)
    x1, x2 = rays[:, 0], rays[:, 1]
    return out + 0.5 * kappa_s * (x1 * x1 + x2 * x2) + 0.5 * gamma * (x1 * x1 - x2 * x2)
