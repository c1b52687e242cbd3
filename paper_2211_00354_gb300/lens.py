"""Thin ctypes binding of liblens.so (include/lens.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Tensors are torch float64 CUDA tensors; the binding passes
their data pointers and the current CUDA stream.  Plan memory comes from the
library's own stream-ordered pool (no Python call per allocation), or, with
use_torch_allocator=True, from torch's caching allocator through the C ABI's
allocator hook.
There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import torch

from . import _build

LENS_OK = 0
LENS_EINVAL = 1
LENS_ENOMEM = 2
LENS_ECUDA = 3
LENS_EDEPTH = 4
LENS_EDOMAIN = 5
LENS_ETIMEOUT = 6
LENS_EFAULT_INJECTED = 7
STATUS_NAMES = {0: "LENS_OK", 1: "LENS_EINVAL", 2: "LENS_ENOMEM", 3: "LENS_ECUDA",
                4: "LENS_EDEPTH", 5: "LENS_EDOMAIN", 6: "LENS_ETIMEOUT",
                7: "LENS_EFAULT_INJECTED"}

FP64 = 0
FP32_BULK = 1
MAP_FUSED = 1
MAP_SEPARATE = 2

# Every symbol include/lens.h declares (checked by the ABI tests).
EXPORTED = ("lens_fmm_build", "lens_deflect", "lens_deflect_grid", "lens_ipm_map",
            "lens_ipm_map_refined", "lens_ipm_map_ex",
            "lens_deflect_adjoint", "lens_plan_info_get", "lens_plan_destroy",
            "lens_direct_deflect", "lens_direct_deflect_noalloc", "lens_light_curve",
            "lens_light_curve_grad", "lens_map_source", "lens_map_histogram", "lens_map_track",
            "lens_find_images", "lens_source_image", "lens_potential",
            "lens_multiplane_deflect", "lens_multiplane_ipm_map",
            "lens_last_error", "lens_version")


class LensError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class lens_build_opts(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("leaf_size", ctypes.c_int), ("prec", ctypes.c_int),
                ("max_depth", ctypes.c_int), ("has_target_box", ctypes.c_int),
                ("target_box", ctypes.c_double * 4)]


class lens_grid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("h", ctypes.c_double),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64)]


class lens_box(ctypes.Structure):
    _fields_ = [("u0", ctypes.c_double), ("u1", ctypes.c_double), ("v0", ctypes.c_double),
                ("v1", ctypes.c_double)]


class lens_ipm_stats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_double), ("area_total", ctypes.c_double),
                ("area_in_map", ctypes.c_double), ("area_outside", ctypes.c_double),
                ("area_dropped", ctypes.c_double), ("area_degenerate", ctypes.c_double),
                ("cells_dropped", ctypes.c_double), ("cells_degenerate", ctypes.c_double),
                ("chunks", ctypes.c_int64), ("ms_deflect", ctypes.c_double),
                ("ms_ipm", ctypes.c_double), ("rays", ctypes.c_double),
                ("p2p_pairs", ctypes.c_double), ("m2p_evals", ctypes.c_double),
                ("ipm_updates", ctypes.c_double), ("cells_queued", ctypes.c_double),
                ("cells_ext", ctypes.c_double),
                ("ms_eval_kernel", ctypes.c_double),
                ("ms_ipm_kernel", ctypes.c_double), ("launches", ctypes.c_int64),
                ("cells_refined", ctypes.c_double), ("fused", ctypes.c_int64),
                ("ms_fused_kernel", ctypes.c_double), ("rays_evaluated", ctypes.c_double)]


class lens_plan_info(ctypes.Structure):
    _fields_ = [("n_stars", ctypes.c_int64), ("n_boxes", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("n_active_boxes", ctypes.c_int64),
                ("n_active_leaves", ctypes.c_int64), ("n_v", ctypes.c_int64),
                ("n_x", ctypes.c_int64), ("n_u", ctypes.c_int64), ("n_w", ctypes.c_int64),
                ("u_stars", ctypes.c_int64), ("levels", ctypes.c_int), ("p", ctypes.c_int),
                ("leaf_size", ctypes.c_int), ("prec", ctypes.c_int),
                ("root_lo", ctypes.c_double * 2), ("root_size", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("ms_build", ctypes.c_double),
                ("build_launches", ctypes.c_int64), ("ms_tree", ctypes.c_double),
                ("ms_far_local", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class lens_plane(ctypes.Structure):
    _fields_ = [("stars_xy", ctypes.c_void_p), ("masses", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("kappa_s", ctypes.c_double), ("gamma", ctypes.c_double)]


class lens_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load liblens.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("liblens.so is missing: run paper_2211_00354_gb300._build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i64, d, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    st = ctypes.c_int
    lib.lens_fmm_build.argtypes = [vp, vp, i64, d, d, ctypes.POINTER(lens_build_opts),
                                   ctypes.POINTER(lens_allocator), vp, ctypes.POINTER(vp)]
    lib.lens_fmm_build.restype = st
    lib.lens_deflect.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.lens_deflect.restype = st
    lib.lens_deflect_grid.argtypes = [vp, ctypes.POINTER(lens_grid), i64, i64, vp, vp, vp]
    lib.lens_deflect_grid.restype = st
    lib.lens_ipm_map.argtypes = [vp, ctypes.POINTER(lens_grid), ctypes.POINTER(lens_box), i, i,
                                 i64, i, vp, ctypes.POINTER(lens_ipm_stats), vp]
    lib.lens_ipm_map.restype = st
    lib.lens_ipm_map_refined.argtypes = [vp, ctypes.POINTER(lens_grid), ctypes.POINTER(lens_box),
                                         i, i, i64, i, i, vp, ctypes.POINTER(lens_ipm_stats), vp]
    lib.lens_ipm_map_refined.restype = st
    lib.lens_ipm_map_ex.argtypes = [vp, ctypes.POINTER(lens_grid), ctypes.POINTER(lens_box),
                                    i, i, i64, i, i, ctypes.c_uint, vp,
                                    ctypes.POINTER(lens_ipm_stats), vp]
    lib.lens_ipm_map_ex.restype = st
    lib.lens_deflect_adjoint.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
    lib.lens_deflect_adjoint.restype = st
    lib.lens_plan_info_get.argtypes = [vp, ctypes.POINTER(lens_plan_info)]
    lib.lens_plan_info_get.restype = st
    lib.lens_plan_destroy.argtypes = [vp]
    lib.lens_plan_destroy.restype = None
    lib.lens_direct_deflect.argtypes = [vp, vp, i64, d, d, vp, i64, i, vp, vp,
                                        ctypes.POINTER(lens_allocator), vp]
    lib.lens_direct_deflect.restype = st
    lib.lens_direct_deflect_noalloc.argtypes = [vp, vp, i64, d, d, vp, i64, vp, vp, vp]
    lib.lens_direct_deflect_noalloc.restype = st
    lib.lens_map_source.argtypes = [vp, i, i, d, d, vp, ctypes.POINTER(lens_allocator), vp]
    lib.lens_map_source.restype = st
    lib.lens_map_histogram.argtypes = [vp, i64, d, d, i, i, vp, vp]
    lib.lens_map_histogram.restype = st
    lib.lens_map_track.argtypes = [vp, i, i, ctypes.POINTER(lens_box), vp, i64, vp, vp]
    lib.lens_map_track.restype = st
    lib.lens_find_images.argtypes = [vp, ctypes.POINTER(lens_grid), d, d, i64, vp, vp,
                                     ctypes.POINTER(ctypes.c_int64), vp]
    lib.lens_find_images.restype = st
    lib.lens_source_image.argtypes = [vp, i64, d, d, d, vp, vp]
    lib.lens_source_image.restype = st
    lib.lens_potential.argtypes = [vp, vp, i64, vp, vp]
    lib.lens_potential.restype = st
    lib.lens_multiplane_deflect.argtypes = [ctypes.POINTER(lens_plane), i, vp,
                                            ctypes.POINTER(lens_build_opts), vp, i64, vp, vp,
                                            ctypes.POINTER(lens_allocator), vp]
    lib.lens_multiplane_deflect.restype = st
    lib.lens_multiplane_ipm_map.argtypes = [ctypes.POINTER(lens_plane), i, vp,
                                            ctypes.POINTER(lens_build_opts),
                                            ctypes.POINTER(lens_grid), ctypes.POINTER(lens_box),
                                            i, i, i64, i, vp, ctypes.POINTER(lens_ipm_stats),
                                            ctypes.POINTER(lens_allocator), vp]
    lib.lens_multiplane_ipm_map.restype = st
    lib.lens_light_curve.argtypes = [vp, i64, d, vp, i64, d, d, vp, vp]
    lib.lens_light_curve.restype = st
    lib.lens_light_curve_grad.argtypes = [vp, i64, d, vp, i64, d, d, vp, vp, vp, vp]
    lib.lens_light_curve_grad.restype = st
    lib.lens_last_error.argtypes = []
    lib.lens_last_error.restype = ctypes.c_char_p
    lib.lens_version.argtypes = []
    lib.lens_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != LENS_OK:
        msg = _lib.lens_last_error().decode(errors="replace")
        raise LensError(status, msg)


def _dev(t: torch.Tensor, name: str, shape_last: Optional[int] = None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (the library has no CPU path)" % name)
    if t.dtype != torch.float64:
        raise TypeError("%s must be float64" % name)
    t = t.contiguous()
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise ValueError("%s must have shape (n, %d)" % (name, shape_last))
    return t


def _stream_ptr(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


# Torch caching-allocator hooks (kept alive at module level).
_live = {}


def _torch_alloc(size, stream, ctx):
    try:
        ptr = torch.cuda.caching_allocator_alloc(int(size), torch.cuda.current_device(),
                                                 int(stream or 0))
        return ptr
    except Exception:  # allocation failure -> NULL -> LENS_ENOMEM
        return None


def _torch_free(ptr, stream, ctx):
    try:
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


_ALLOC_CB = ALLOC_FN(_torch_alloc)
_FREE_CB = FREE_FN(_torch_free)
TORCH_ALLOCATOR = lens_allocator(_ALLOC_CB, _FREE_CB, None)


def grid_struct(grid) -> lens_grid:
    return lens_grid(float(grid.x0), float(grid.y0), float(grid.h), int(grid.nx), int(grid.ny))


class LensFMM:
    """An FMM plan over a star field (lens_fmm_build) and its evaluations."""

    def __init__(self, stars: torch.Tensor, masses: torch.Tensor, kappa_s: float = 0.0,
                 gamma: float = 0.0, p: int = 16, leaf_size: int = 16, prec: int = FP32_BULK,
                 target_box=None, max_depth: int = 0, use_torch_allocator: bool = False,
                 stream=None):
        lib = load()
        stars = _dev(stars, "stars", 2)
        masses = _dev(masses, "masses").reshape(-1)
        if masses.shape[0] != stars.shape[0]:
            raise ValueError("stars and masses disagree in length")
        opts = lens_build_opts()
        opts.p, opts.leaf_size, opts.prec, opts.max_depth = int(p), int(leaf_size), int(prec), int(max_depth)
        if target_box is not None:
            opts.has_target_box = 1
            for k in range(4):
                opts.target_box[k] = float(target_box[k])
        self._handle = ctypes.c_void_p()
        self.kappa_s, self.gamma, self.p, self.leaf_size, self.prec = (
            float(kappa_s), float(gamma), int(p), int(leaf_size), int(prec))
        self.n = int(stars.shape[0])
        alloc = ctypes.byref(TORCH_ALLOCATOR) if use_torch_allocator else None
        self._stars, self._masses = stars, masses  # kept alive until the build syncs
        _check(lib.lens_fmm_build(stars.data_ptr(), masses.data_ptr(), self.n, self.kappa_s,
                                  self.gamma, ctypes.byref(opts), alloc, _stream_ptr(stream),
                                  ctypes.byref(self._handle)))
        self._stars = self._masses = None

    def close(self):
        if getattr(self, "_handle", None) is not None and self._handle.value:
            _lib.lens_plan_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self) -> dict:
        inf = lens_plan_info()
        _check(_lib.lens_plan_info_get(self._handle, ctypes.byref(inf)))
        out = {}
        for name, _ in lens_plan_info._fields_:
            v = getattr(inf, name)
            out[name] = list(v) if name == "root_lo" else v
        return out

    def deflect(self, rays: torch.Tensor, jacobian: bool = False, stream=None):
        rays = _dev(rays, "rays", 2)
        m = rays.shape[0]
        y = torch.empty_like(rays)
        jac = torch.empty((m, 2, 2), dtype=torch.float64, device=rays.device) if jacobian else None
        _check(_lib.lens_deflect(self._handle, rays.data_ptr(), m, y.data_ptr(),
                                 jac.data_ptr() if jacobian else None, _stream_ptr(stream)))
        return (y, jac) if jacobian else y

    def potential(self, rays: torch.Tensor, stream=None):
        """Lensing potential psi at rays (m x 2) (lens_potential)."""
        rays = _dev(rays, "rays", 2)
        psi = torch.empty((rays.shape[0],), dtype=torch.float64, device=rays.device)
        _check(_lib.lens_potential(self._handle, rays.data_ptr(), rays.shape[0], psi.data_ptr(),
                                   _stream_ptr(stream)))
        return psi

    def deflect_grid(self, grid, row0: int = 0, nrows: Optional[int] = None,
                     jacobian: bool = False, stream=None):
        g = grid_struct(grid)
        if nrows is None:
            nrows = g.ny + 1 - row0
        dev = torch.device("cuda", torch.cuda.current_device())
        y = torch.empty((nrows, g.nx + 1, 2), dtype=torch.float64, device=dev)
        jac = (torch.empty((nrows, g.nx + 1, 2, 2), dtype=torch.float64, device=dev)
               if jacobian else None)
        _check(_lib.lens_deflect_grid(self._handle, ctypes.byref(g), int(row0), int(nrows),
                                      y.data_ptr(), jac.data_ptr() if jacobian else None,
                                      _stream_ptr(stream)))
        return (y, jac) if jacobian else y

    def ipm_map(self, grid, box, npx: int, npy: int, max_cells_per_chunk: int = 0,
                bbox_cap: int = 0, out: Optional[torch.Tensor] = None, stream=None,
                refine_levels: int = 0, fused: Optional[bool] = None):
        """Magnification map (lens_ipm_map_ex: refine_levels > 0 splits cells
        over bbox_cap 2 x 2 instead of dropping them; fused True / False picks
        the fused deflection + IPM kernel or the separate kernels, None the
        library's default)."""
        g = grid_struct(grid)
        b = lens_box(*(float(v) for v in box))
        dev = torch.device("cuda", torch.cuda.current_device())
        mp = out if out is not None else torch.empty((npy, npx), dtype=torch.float64, device=dev)
        st = lens_ipm_stats()
        flags = 0 if fused is None else (MAP_FUSED if fused else MAP_SEPARATE)
        _check(_lib.lens_ipm_map_ex(self._handle, ctypes.byref(g), ctypes.byref(b), int(npx),
                                    int(npy), int(max_cells_per_chunk), int(bbox_cap),
                                    int(refine_levels), flags, mp.data_ptr(), ctypes.byref(st),
                                    _stream_ptr(stream)))
        stats = {name: getattr(st, name) for name, _ in lens_ipm_stats._fields_}
        return mp, stats

    def adjoint(self, rays: torch.Tensor, grad_y: torch.Tensor, stream=None):
        rays = _dev(rays, "rays", 2)
        grad_y = _dev(grad_y, "grad_y", 2)
        dev = rays.device
        gxy = torch.empty((self.n, 2), dtype=torch.float64, device=dev)
        gm = torch.empty((self.n,), dtype=torch.float64, device=dev)
        gkg = torch.empty((2,), dtype=torch.float64, device=dev)
        _check(_lib.lens_deflect_adjoint(self._handle, rays.data_ptr(), rays.shape[0],
                                         grad_y.data_ptr(), gxy.data_ptr(), gm.data_ptr(),
                                         gkg.data_ptr(), _stream_ptr(stream)))
        return gxy, gm, gkg


def _planes(planes, beta):
    """(lens_plane array, kept tensors, beta as a contiguous host buffer)."""
    K = len(planes)
    arr = (lens_plane * K)()
    keep = []
    for k, (st, ms, ks, g) in enumerate(planes):
        st = _dev(st, "stars", 2)
        ms = _dev(ms, "masses").reshape(-1)
        if ms.shape[0] != st.shape[0]:
            raise ValueError("a plane's stars and masses disagree in length")
        keep += [st, ms]
        arr[k] = lens_plane(st.data_ptr() if st.shape[0] else None,
                            ms.data_ptr() if ms.shape[0] else None, int(st.shape[0]),
                            float(ks), float(g))
    b = (ctypes.c_double * (K * K))()
    rows = [list(map(float, r)) for r in beta]
    if len(rows) != K or any(len(r) != K for r in rows):
        raise ValueError("beta must be nplanes x nplanes")
    for i in range(K):
        for j in range(K):
            b[i * K + j] = rows[i][j]
    return arr, keep, b


def _mp_opts(p, leaf_size, prec, max_depth=0):
    o = lens_build_opts()
    o.p, o.leaf_size, o.prec, o.max_depth = int(p), int(leaf_size), int(prec), int(max_depth)
    return o


def multiplane_deflect(planes, beta, rays, p=16, leaf_size=16, prec=FP32_BULK,
                       planes_out=False, stream=None):
    """Rays through several lens planes (lens_multiplane_deflect).  planes: a
    list of (stars (n, 2), masses (n,), kappa_s, gamma) CUDA float64 tensors
    and floats, nearest first; beta: nplanes x nplanes distance ratios.
    Returns y (m, 2) [, x_planes (nplanes, m, 2)]."""
    lib = load()
    rays = _dev(rays, "rays", 2)
    arr, keep, b = _planes(planes, beta)
    K = len(planes)
    y = torch.empty_like(rays)
    xp = (torch.empty((K, rays.shape[0], 2), dtype=torch.float64, device=rays.device)
          if planes_out else None)
    o = _mp_opts(p, leaf_size, prec)
    _check(lib.lens_multiplane_deflect(arr, K, ctypes.cast(b, ctypes.c_void_p), ctypes.byref(o),
                                       rays.data_ptr(), rays.shape[0], y.data_ptr(),
                                       xp.data_ptr() if planes_out else None, None,
                                       _stream_ptr(stream)))
    return (y, xp) if planes_out else y


def multiplane_ipm_map(planes, beta, grid, box, npx, npy, p=16, leaf_size=16, prec=FP32_BULK,
                       max_cells_per_chunk=0, bbox_cap=0, out=None, stream=None):
    """Magnification map through several lens planes (lens_multiplane_ipm_map)."""
    lib = load()
    arr, keep, b = _planes(planes, beta)
    g = grid_struct(grid)
    bx = lens_box(*(float(v) for v in box))
    dev = torch.device("cuda", torch.cuda.current_device())
    mp = out if out is not None else torch.empty((npy, npx), dtype=torch.float64, device=dev)
    st = lens_ipm_stats()
    o = _mp_opts(p, leaf_size, prec)
    _check(lib.lens_multiplane_ipm_map(arr, len(planes), ctypes.cast(b, ctypes.c_void_p),
                                       ctypes.byref(o), ctypes.byref(g), ctypes.byref(bx),
                                       int(npx), int(npy), int(max_cells_per_chunk),
                                       int(bbox_cap), mp.data_ptr(), ctypes.byref(st), None,
                                       _stream_ptr(stream)))
    return mp, {name: getattr(st, name) for name, _ in lens_ipm_stats._fields_}


def direct_deflect(stars, masses, kappa_s, gamma, rays, prec=FP64, jacobian=False, stream=None):
    """Eq. 1 by GPU direct summation (lens_direct_deflect)."""
    lib = load()
    stars = _dev(stars, "stars", 2)
    masses = _dev(masses, "masses").reshape(-1)
    rays = _dev(rays, "rays", 2)
    y = torch.empty_like(rays)
    jac = torch.empty((rays.shape[0], 2, 2), dtype=torch.float64, device=rays.device) if jacobian else None
    _check(lib.lens_direct_deflect(stars.data_ptr(), masses.data_ptr(), stars.shape[0],
                                   float(kappa_s), float(gamma), rays.data_ptr(), rays.shape[0],
                                   int(prec), y.data_ptr(), jac.data_ptr() if jacobian else None,
                                   ctypes.byref(TORCH_ALLOCATOR), _stream_ptr(stream)))
    return (y, jac) if jacobian else y


NOALLOC_MAX_STARS = 1 << 18


def direct_deflect_noalloc(stars, masses, kappa_s, gamma, rays, jacobian=False, out=None,
                           stream=None):
    """Float32 direct sum through lens_direct_deflect_noalloc: the library
    allocates no device memory for it (fixed static scratch, <= 262144 stars).
    Pass ``out`` (m, 2) to avoid even the output allocation on this side."""
    lib = load()
    stars = _dev(stars, "stars", 2)
    masses = _dev(masses, "masses").reshape(-1)
    rays = _dev(rays, "rays", 2)
    y = out if out is not None else torch.empty_like(rays)
    jac = torch.empty((rays.shape[0], 2, 2), dtype=torch.float64, device=rays.device) if jacobian else None
    _check(lib.lens_direct_deflect_noalloc(stars.data_ptr(), masses.data_ptr(), stars.shape[0],
                                           float(kappa_s), float(gamma), rays.data_ptr(),
                                           rays.shape[0], y.data_ptr(),
                                           jac.data_ptr() if jacobian else None,
                                           _stream_ptr(stream)))
    return (y, jac) if jacobian else y


def map_source(mp, sigma_px, trunc=6.0, stream=None):
    """The map seen by a Gaussian source of sigma_px pixels (lens_map_source)."""
    lib = load()
    mp = _dev(mp, "map")
    out = torch.empty_like(mp)
    _check(lib.lens_map_source(mp.data_ptr(), mp.shape[1], mp.shape[0], float(sigma_px),
                               float(trunc), out.data_ptr(), None, _stream_ptr(stream)))
    return out


def map_histogram(values, lo, hi, nbins, log_bins=False, stream=None):
    """counts[0] below lo, counts[1..nbins] the bins, counts[nbins+1] above
    (lens_map_histogram)."""
    lib = load()
    v = _dev(values, "values").reshape(-1)
    counts = torch.empty((nbins + 2,), dtype=torch.int64, device=v.device)
    _check(lib.lens_map_histogram(v.data_ptr(), v.shape[0], float(lo), float(hi), int(nbins),
                                  int(bool(log_bins)), counts.data_ptr(), _stream_ptr(stream)))
    return counts


def map_track(mp, box, positions, stream=None):
    """The map at source positions (k x 2), bilinear (lens_map_track)."""
    lib = load()
    mp = _dev(mp, "map")
    pos = _dev(positions, "positions", 2)
    out = torch.empty((pos.shape[0],), dtype=torch.float64, device=mp.device)
    b = lens_box(*(float(v) for v in box))
    _check(lib.lens_map_track(mp.data_ptr(), mp.shape[1], mp.shape[0], ctypes.byref(b),
                              pos.data_ptr(), pos.shape[0], out.data_ptr(), _stream_ptr(stream)))
    return out


def find_images(y, grid, beta, max_out=64, stream=None):
    """Images of the point source beta on a deflected grid (lens_find_images):
    y (ny+1, nx+1, 2) as deflect_grid returns it.  Returns (cells int64 [k],
    images float64 [k, 3] = x1, x2, signed magnification), sorted by cell."""
    lib = load()
    y = _dev(y.reshape(-1, 2), "y", 2)
    if y.shape[0] != (grid.nx + 1) * (grid.ny + 1):
        raise ValueError("y must hold the (nx+1) x (ny+1) corners of the grid")
    g = grid_struct(grid)
    while True:
        out = torch.empty((max(max_out, 1), 3), dtype=torch.float64, device=y.device)
        cells = torch.empty((max(max_out, 1),), dtype=torch.int64, device=y.device)
        n = ctypes.c_int64(0)
        _check(lib.lens_find_images(y.data_ptr(), ctypes.byref(g), float(beta[0]), float(beta[1]),
                                    max_out, out.data_ptr(), cells.data_ptr(), ctypes.byref(n),
                                    _stream_ptr(stream)))
        if n.value <= max_out:
            break
        max_out = n.value
    cells, out = cells[:n.value], out[:n.value]
    order = torch.argsort(cells)
    return cells[order], out[order]


def source_image(y, beta, sigma, stream=None):
    """exp(-|y - beta|^2 / 2 sigma^2) at every ray (lens_source_image)."""
    lib = load()
    shape = y.shape[:-1]
    y = _dev(y.reshape(-1, 2), "y", 2)
    out = torch.empty((y.shape[0],), dtype=torch.float64, device=y.device)
    _check(lib.lens_source_image(y.data_ptr(), y.shape[0], float(beta[0]), float(beta[1]),
                                 float(sigma), out.data_ptr(), _stream_ptr(stream)))
    return out.reshape(shape)


def light_curve(y, w_ray, samples, sigma, trunc=6.0, stream=None):
    lib = load()
    y = _dev(y.reshape(-1, 2), "y", 2)
    samples = _dev(samples, "samples", 2)
    F = torch.empty((samples.shape[0],), dtype=torch.float64, device=y.device)
    _check(lib.lens_light_curve(y.data_ptr(), y.shape[0], float(w_ray), samples.data_ptr(),
                                samples.shape[0], float(sigma), float(trunc), F.data_ptr(),
                                _stream_ptr(stream)))
    return F


def light_curve_grad(y, w_ray, samples, sigma, F, T, trunc=6.0, stream=None):
    lib = load()
    y = _dev(y.reshape(-1, 2), "y", 2)
    samples = _dev(samples, "samples", 2)
    F = _dev(F, "F")
    T = _dev(T, "T")
    g = torch.empty_like(y)
    _check(lib.lens_light_curve_grad(y.data_ptr(), y.shape[0], float(w_ray), samples.data_ptr(),
                                     samples.shape[0], float(sigma), float(trunc), F.data_ptr(),
                                     T.data_ptr(), g.data_ptr(), _stream_ptr(stream)))
    return g


def version() -> str:
    return load().lens_version().decode()
