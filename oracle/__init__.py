"""FP64 CPU oracle for the FMM-IPM hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from it: the two share no code.  Inputs come
from the seeded generators in ``paper_2211_00354_gb300.synth`` (which hold
none of the method's arithmetic) or are written here by hand.

Routines (all plain definitions; see the header of ``lens_oracle.c``):

* :func:`deflect` -- Eq. 1 direct sum with kappa_s, gamma (footnote to Eq. 1).
* :func:`ipm_map` -- first-order IPM (Sec. 2.3, step 4 of the Sec. 2.4
  algorithm) with a flux ledger.
* :func:`clip_area_sh`, :func:`clip_area_green` -- two independent
  polygon/pixel overlap routines (Green's theorem apportioning, Sec. 2.3).
* :func:`adjoint` -- gradient through Eq. 1 from its real-variable derivatives.
* :func:`light_curve`, :func:`light_curve_grad` -- Gaussian-source light
  curve as a ray sum (light curves: Sec. 3.3; Gaussian source: Sec. 2.5).
* :func:`find_images`, :func:`source_image` (``images.py``) -- images of a
  point source as the grid cells whose deflected quadrilateral winds around
  it, located by inverting the cell's bilinear map, and the lensed image of
  a Gaussian source (Sec. 2.5).
* :func:`potential` (``potential.py``) -- the lensing potential
  sum m ln|x - x_i| + smooth field, by direct sum (Sec. 2.5).

Parity unpinned: none -- every routine has closed-form or brute-force pins in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .images import find_images, source_image, winding_numbers  # noqa: F401
from .potential import potential  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lens_oracle.c")
_LIB = os.path.join(_HERE, "liblens_oracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``lens_oracle.c`` with gcc (OpenMP) into ``liblens_oracle.so``."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64 = ctypes.c_int64
        d = ctypes.c_double
        lib.oracle_deflect.argtypes = [i64, _dp, _dp, d, d, i64, _dp, _dp, _dp, _dp]
        lib.oracle_deflect.restype = None
        lib.oracle_clip_area_sh.argtypes = [_dp, ctypes.c_int, d, d]
        lib.oracle_clip_area_sh.restype = d
        lib.oracle_clip_area_green.argtypes = [_dp, ctypes.c_int, d, d]
        lib.oracle_clip_area_green.restype = d
        lib.oracle_ipm_map.argtypes = [i64, i64, d, _dp, d, d, d, d, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, _dp, _dp]
        lib.oracle_ipm_map.restype = None
        lib.oracle_ipm_map_refined.argtypes = [i64, i64, d, d, d, _dp, i64, _dp, _dp, d, d, d, d,
                                               d, d, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, _dp, _dp]
        lib.oracle_ipm_map_refined.restype = None
        ci = ctypes.c_int
        lib.oracle_multiplane_deflect.argtypes = [ci, ctypes.POINTER(i64),
                                                  ctypes.POINTER(_dp), ctypes.POINTER(_dp),
                                                  _dp, _dp, _dp, i64, _dp, _dp, _dp]
        lib.oracle_multiplane_deflect.restype = None
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ci
        lib.oracle_map_convolve_gaussian.argtypes = [ci, ci, _dp, d, d, _dp]
        lib.oracle_map_convolve_gaussian.restype = None
        lib.oracle_histogram.argtypes = [i64, _dp, d, d, ci, ci, ctypes.POINTER(i64)]
        lib.oracle_histogram.restype = None
        lib.oracle_map_track.argtypes = [ci, ci, _dp, d, d, d, d, i64, _dp, _dp]
        lib.oracle_map_track.restype = None
        lib.oracle_adjoint.argtypes = [i64, _dp, _dp, i64, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_adjoint.restype = None
        lib.oracle_light_curve.argtypes = [i64, _dp, d, i64, _dp, d, d, _dp]
        lib.oracle_light_curve.restype = None
        lib.oracle_light_curve_grad.argtypes = [i64, _dp, d, i64, _dp, d, d, _dp, _dp, _dp]
        lib.oracle_light_curve_grad.restype = None
        _lib = lib
    return _lib


def threads() -> int:
    """Threads the oracle's OpenMP loops run on."""
    return int(_load().oracle_threads())


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def deflect(stars, masses, kappa_s, gamma, rays, *, alpha=False, jacobian=False):
    """Eq. 1 by direct summation.  Returns y (m, 2) [, alpha (m, 2)] [, jac (m, 2, 2)]."""
    lib = _load()
    stars, ps = _c(np.asarray(stars).reshape(-1, 2))
    masses, pm = _c(np.asarray(masses).reshape(-1))
    rays, pr = _c(np.asarray(rays).reshape(-1, 2))
    n, m = stars.shape[0], rays.shape[0]
    assert masses.shape[0] == n
    y = np.empty((m, 2))
    al = np.empty((m, 2)) if alpha else None
    jac = np.empty((m, 2, 2)) if jacobian else None
    lib.oracle_deflect(n, ps, pm, float(kappa_s), float(gamma), m, pr,
                       y.ctypes.data_as(_dp),
                       al.ctypes.data_as(_dp) if alpha else None,
                       jac.ctypes.data_as(_dp) if jacobian else None)
    out = [y]
    if alpha:
        out.append(al)
    if jacobian:
        out.append(jac)
    return out[0] if len(out) == 1 else tuple(out)


def multiplane_deflect(planes, beta, rays, *, planes_out=False):
    """Rays through K thin lens planes.  planes: K tuples (stars (n, 2),
    masses (n,), kappa_s, gamma); beta: (K, K), beta[i, j] for i < j the
    distance ratio of planes i and j.  Returns y (m, 2) [, x_planes (K, m, 2)]."""
    lib = _load()
    K = len(planes)
    keep = []
    ns = (ctypes.c_int64 * K)()
    sp = (_dp * K)()
    mp = (_dp * K)()
    kap = np.empty(K)
    gam = np.empty(K)
    for i, (st, ms, ks, g) in enumerate(planes):
        st, pst = _c(np.asarray(st, dtype=np.float64).reshape(-1, 2))
        ms, pms = _c(np.asarray(ms, dtype=np.float64).reshape(-1))
        assert ms.shape[0] == st.shape[0]
        keep += [st, ms]
        ns[i] = st.shape[0]
        sp[i] = pst
        mp[i] = pms
        kap[i], gam[i] = float(ks), float(g)
    b, pb = _c(np.asarray(beta, dtype=np.float64).reshape(K, K))
    rays, pr = _c(np.asarray(rays).reshape(-1, 2))
    m = rays.shape[0]
    y = np.empty((m, 2))
    xp = np.empty((K, m, 2)) if planes_out else None
    lib.oracle_multiplane_deflect(K, ns, sp, mp, kap.ctypes.data_as(_dp), gam.ctypes.data_as(_dp),
                                  pb, m, pr, y.ctypes.data_as(_dp),
                                  xp.ctypes.data_as(_dp) if planes_out else None)
    return (y, xp) if planes_out else y


def clip_area_sh(poly, x0, y0):
    """Signed overlap of a polygon with the unit square at (x0, y0): Sutherland-Hodgman."""
    lib = _load()
    p, pp = _c(np.asarray(poly).reshape(-1, 2))
    assert p.shape[0] <= 16
    return lib.oracle_clip_area_sh(pp, p.shape[0], float(x0), float(y0))


def clip_area_green(poly, x0, y0):
    """Signed overlap of a polygon with the unit square at (x0, y0): Green's theorem."""
    lib = _load()
    p, pp = _c(np.asarray(poly).reshape(-1, 2))
    return lib.oracle_clip_area_green(pp, p.shape[0], float(x0), float(y0))


IPM_STAT_KEYS = ("cells", "area_total", "area_in_map", "area_outside",
                 "area_dropped", "area_degenerate", "cells_dropped",
                 "cells_degenerate")


def ipm_map(ycorn, h, box, npx, npy, bbox_cap=0):
    """First-order IPM of a grid of deflected corners.

    ycorn: (ny+1, nx+1, 2) deflected corner positions; h: cell side;
    box: (u0, u1, v0, v1) source-plane window; returns (map (npy, npx), stats dict).
    """
    lib = _load()
    yc, py_ = _c(ycorn)
    assert yc.ndim == 3 and yc.shape[2] == 2
    ny, nx = yc.shape[0] - 1, yc.shape[1] - 1
    mp = np.empty((npy, npx))
    st = np.empty(8)
    u0, u1, v0, v1 = (float(v) for v in box)
    lib.oracle_ipm_map(nx, ny, float(h), py_, u0, u1, v0, v1, int(npx), int(npy),
                       int(bbox_cap), mp.ctypes.data_as(_dp), st.ctypes.data_as(_dp))
    return mp, dict(zip(IPM_STAT_KEYS, st.tolist()))


def ipm_map_refined(ycorn, x0, y0, h, stars, masses, kappa_s, gamma, box, npx, npy, bbox_cap,
                    levels):
    """IPM with critical-cell refinement: cells whose pixel box exceeds
    bbox_cap are split 2 x 2 (new corners by the direct sum) up to `levels`
    times.  ycorn: (ny+1, nx+1, 2) deflected corners of the grid whose cell
    (i, j) starts at (x0 + i h, y0 + j h).  Returns (map, stats dict)."""
    lib = _load()
    yc, py_ = _c(ycorn)
    assert yc.ndim == 3 and yc.shape[2] == 2
    ny, nx = yc.shape[0] - 1, yc.shape[1] - 1
    st_, sp = _c(np.asarray(stars).reshape(-1, 2))
    ms, mp_ = _c(np.asarray(masses).reshape(-1))
    mp = np.empty((npy, npx))
    st = np.empty(8)
    u0, u1, v0, v1 = (float(v) for v in box)
    lib.oracle_ipm_map_refined(nx, ny, float(x0), float(y0), float(h), py_, st_.shape[0], sp, mp_,
                               float(kappa_s), float(gamma), u0, u1, v0, v1, int(npx), int(npy),
                               int(bbox_cap), int(levels), mp.ctypes.data_as(_dp),
                               st.ctypes.data_as(_dp))
    return mp, dict(zip(IPM_STAT_KEYS, st.tolist()))


def map_convolve_gaussian(mp, sigma_px, trunc=6.0):
    """The map seen by a circular Gaussian source of sigma_px pixels (the
    profile cut at the isophote |d| = trunc sigma, renormalised to its part
    inside the map)."""
    lib = _load()
    m, mp_ = _c(mp)
    out = np.empty_like(m)
    lib.oracle_map_convolve_gaussian(m.shape[1], m.shape[0], mp_, float(sigma_px), float(trunc),
                                     out.ctypes.data_as(_dp))
    return out


def histogram(v, lo, hi, nbins, log_bins=False):
    """counts[0] below lo, counts[1..nbins] the bins, counts[nbins+1] above."""
    lib = _load()
    a, ap = _c(np.asarray(v).reshape(-1))
    counts = np.zeros(nbins + 2, dtype=np.int64)
    lib.oracle_histogram(a.shape[0], ap, float(lo), float(hi), int(nbins), int(bool(log_bins)),
                         counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return counts


def map_track(mp, box, s):
    """The map at source positions s (k x 2), bilinear between pixel centres."""
    lib = _load()
    m, mp_ = _c(mp)
    ss, sp = _c(np.asarray(s).reshape(-1, 2))
    out = np.empty(ss.shape[0])
    u0, u1, v0, v1 = (float(x) for x in box)
    lib.oracle_map_track(m.shape[1], m.shape[0], mp_, u0, u1, v0, v1, ss.shape[0], sp,
                         out.ctypes.data_as(_dp))
    return out


def adjoint(stars, masses, rays, grad_y):
    """Gradient through Eq. 1: returns (d/dstars (n,2), d/dmasses (n,), [d/dkappa_s, d/dgamma])."""
    lib = _load()
    stars, ps = _c(np.asarray(stars).reshape(-1, 2))
    masses, pm = _c(np.asarray(masses).reshape(-1))
    rays, pr = _c(np.asarray(rays).reshape(-1, 2))
    gy, pg = _c(np.asarray(grad_y).reshape(-1, 2))
    n, m = stars.shape[0], rays.shape[0]
    gxy = np.empty((n, 2))
    gm = np.empty(n)
    gkg = np.empty(2)
    lib.oracle_adjoint(n, ps, pm, m, pr, pg, gxy.ctypes.data_as(_dp),
                       gm.ctypes.data_as(_dp), gkg.ctypes.data_as(_dp))
    return gxy, gm, gkg


def light_curve(y, w_ray, samples, sigma, trunc=6.0):
    """F_k = sum_r w_ray G_sigma(y_r - s_k), G a unit-normalised 2-D Gaussian cut at trunc*sigma."""
    lib = _load()
    y, pyy = _c(np.asarray(y).reshape(-1, 2))
    s, ps = _c(np.asarray(samples).reshape(-1, 2))
    F = np.empty(s.shape[0])
    lib.oracle_light_curve(y.shape[0], pyy, float(w_ray), s.shape[0], ps,
                           float(sigma), float(trunc), F.ctypes.data_as(_dp))
    return F


def light_curve_grad(y, w_ray, samples, sigma, F, T, trunc=6.0):
    """dL/dy for L = sum_k (F_k - T_k)^2."""
    lib = _load()
    y, pyy = _c(np.asarray(y).reshape(-1, 2))
    s, ps = _c(np.asarray(samples).reshape(-1, 2))
    F, pF = _c(F)
    T, pT = _c(T)
    g = np.empty_like(y)
    lib.oracle_light_curve_grad(y.shape[0], pyy, float(w_ray), s.shape[0], ps,
                                float(sigma), float(trunc), pF, pT,
                                g.ctypes.data_as(_dp))
    return g


def light_curve_loss(y, w_ray, samples, sigma, T, trunc=6.0):
    F = light_curve(y, w_ray, samples, sigma, trunc)
    return float(np.sum((F - np.asarray(T)) ** 2)), F
