"""Seeded synthetic workloads shaped like the paper's lens fields.

This module feeds both the CUDA path and the CPU oracle, so it holds none of
the method's arithmetic: only random star fields, masses, ray grids and map
windows.  Every generator takes an explicit seed (numpy ``default_rng``).

Shapes follow the paper's workloads: uniform circular star fields circumscribing
the shooting region (Sec. 2.3, 2D shell theorem), clustered primordial black
holes (Sec. 3.2), a strongly anamorphic region near a critical curve (Sec. 3.3)
and a many-particle halo (Sec. 2.5).  The paper's own datasets (EAGLE halo,
figure data) are not available; these generators stand in for them.

Conventions: Einstein units; kappa_* of a uniform disk of radius R holding
point masses m_i is sum(m_i)/R^2.  The smooth field is y1 = (1-ks-g) x1 - a1,
y2 = (1-ks+g) x2 - a2, so a map of half-size L/2 needs rays over
|x1| <= (L/2)/|1-k-g| and |x2| <= (L/2)/|1-k+g| (k = ks + kappa_*), plus a
margin.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np


@dataclasses.dataclass
class Grid:
    """Image-plane cell grid: cells [x0 + i h, x0 + (i+1) h) x [y0 + j h, ...).

    nx x ny cells, (nx+1) x (ny+1) corner rays.
    """
    x0: float
    y0: float
    h: float
    nx: int
    ny: int

    @property
    def n_rays(self) -> int:
        return (self.nx + 1) * (self.ny + 1)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny

    def corners(self) -> np.ndarray:
        """(ny+1, nx+1, 2) corner positions, computed as x0 + i*h (the same
        expression the library evaluates)."""
        i = np.arange(self.nx + 1, dtype=np.float64)
        j = np.arange(self.ny + 1, dtype=np.float64)
        X = self.x0 + i * self.h
        Y = self.y0 + j * self.h
        out = np.empty((self.ny + 1, self.nx + 1, 2))
        out[..., 0] = X[None, :]
        out[..., 1] = Y[:, None]
        return out


@dataclasses.dataclass
class Field:
    stars: np.ndarray      # (n, 2) float64
    masses: np.ndarray     # (n,)  float64
    kappa_s: float
    gamma: float
    kappa_star: float
    grid: Optional[Grid] = None
    box: Optional[Tuple[float, float, float, float]] = None  # map window u0,u1,v0,v1
    npx: int = 0
    npy: int = 0
    name: str = ""

    @property
    def n(self) -> int:
        return self.stars.shape[0]


def uniform_disk(rng: np.random.Generator, n: int, radius: float,
                 center=(0.0, 0.0)) -> np.ndarray:
    r = radius * np.sqrt(rng.random(n))
    t = 2.0 * math.pi * rng.random(n)
    out = np.empty((n, 2))
    out[:, 0] = center[0] + r * np.cos(t)
    out[:, 1] = center[1] + r * np.sin(t)
    return out


def shooting_grid(kappa: float, gamma: float, half_map: float, h: float,
                  margin_frac: float = 0.03, margin_min: float = 0.0,
                  half_extent: Optional[Tuple[float, float]] = None) -> Grid:
    """Cell grid covering the image-plane region that maps onto a square map of
    half-size ``half_map`` (plus a margin), with cell side h."""
    if half_extent is None:
        e1 = half_map / abs(1.0 - kappa - gamma)
        e2 = half_map / abs(1.0 - kappa + gamma)
        e1 += max(margin_frac * e1, margin_min)
        e2 += max(margin_frac * e2, margin_min)
    else:
        e1, e2 = half_extent
    nx = int(math.ceil(2 * e1 / h))
    ny = int(math.ceil(2 * e2 / h))
    return Grid(x0=-0.5 * nx * h, y0=-0.5 * ny * h, h=h, nx=nx, ny=ny)


def config_uniform(seed: int, n: int, kappa_star: float, kappa_s: float,
                   gamma: float, mass_range=None, radius: Optional[float] = None,
                   name: str = "") -> Field:
    rng = np.random.default_rng(seed)
    if mass_range is None:
        m = np.ones(n)
    else:
        m = rng.uniform(mass_range[0], mass_range[1], n)
    if radius is None:
        radius = math.sqrt(float(np.sum(m)) / kappa_star)
    stars = uniform_disk(rng, n, radius)
    return Field(stars=stars, masses=m, kappa_s=kappa_s, gamma=gamma,
                 kappa_star=kappa_star, name=name)


# ---------------------------------------------------------------------------
# Named workloads (sizes scale down with ``scale`` for tests that need the
# oracle to finish in seconds; scale=1 is the full workload).

def c1_plain(seed: int = 0) -> Field:
    """1e3 equal-mass stars, kappa_*=0.4, no smooth field; 500^2 cells over the
    central 20x20 ER; 100^2-pixel map over 10x10 ER."""
    f = config_uniform(seed, 1000, 0.4, 0.0, 0.0, name="c1-plain-1e3")
    f.grid = Grid(x0=-10.0, y0=-10.0, h=0.04, nx=500, ny=500)
    f.box = (-5.0, 5.0, -5.0, 5.0)
    f.npx = f.npy = 100
    return f


def c2_high_mag(seed: int = 0, n: int = 1_500_000, npix: int = 2000,
                half_map: float = 100.0, h: float = 0.063) -> Field:
    """High-magnification map: kappa_*=0.45, kappa_s=0, gamma=0.45 (mu=10);
    N*=1.5e6 equal-mass stars uniform in a disk of radius sqrt(N*/kappa_*);
    map 2000^2 pixels over 200 ER; ~1e8 cells (h = 0.063 ER)."""
    f = config_uniform(seed, n, 0.45, 0.0, 0.45, name="c2-highmag")
    f.grid = shooting_grid(0.45, 0.45, half_map, h, margin_frac=0.03,
                           margin_min=max(10.0 * h, 0.1 * half_map))
    f.box = (-half_map, half_map, -half_map, half_map)
    f.npx = f.npy = npix
    return f


def c2_window(seed: int = 0, npix: int = 200, h: float = 0.063) -> Field:
    """A window of the high-magnification map: npix^2 pixels of 0.1 ER
    (kappa_*=0.45, kappa_s=0, gamma=0.45, cells of side h), its shooting
    region alone, equal-mass stars uniform in a disk that circumscribes that
    region with a quarter of its radius to spare (star density kappa_*, as in
    the full map)."""
    half = 0.05 * npix
    grid = shooting_grid(0.45, 0.45, half, h, margin_frac=0.03, margin_min=max(10.0 * h, 0.1 * half))
    rc = math.hypot(0.5 * grid.nx * h, 0.5 * grid.ny * h)
    n = int(math.ceil(0.45 * (1.25 * rc) ** 2))
    f = config_uniform(seed, n, 0.45, 0.0, 0.45, name="c2-window")
    f.grid = grid
    f.box = (-half, half, -half, half)
    f.npx = f.npy = npix
    return f


def c3_clustered(seed: int = 0, n_clusters: int = 1000, per_cluster: int = 1000,
                 a: float = 0.5, npix: int = 4096, half_map: float = 50.0,
                 h: float = 0.0244, trunc: float = 20.0) -> Field:
    """Clustered PBH field: Plummer clusters (scale a, projected radius
    R = a sqrt(u/(1-u)), truncated at trunc*a), cluster centres uniform in a
    disk; masses log-normal (median 1, sigma_ln = 1); kappa_*=0.2,
    kappa_s=0.3, gamma=0.3."""
    rng = np.random.default_rng(seed)
    n = n_clusters * per_cluster
    m = rng.lognormal(0.0, 1.0, n)
    kappa_star = 0.2
    radius = math.sqrt(float(np.sum(m)) / kappa_star)
    centres = uniform_disk(rng, n_clusters, radius)
    u = rng.random(n)
    rmax2 = trunc * trunc
    umax = rmax2 / (1.0 + rmax2)
    u = u * umax
    rr = a * np.sqrt(u / (1.0 - u))
    t = 2.0 * math.pi * rng.random(n)
    stars = np.repeat(centres, per_cluster, axis=0)
    stars[:, 0] += rr * np.cos(t)
    stars[:, 1] += rr * np.sin(t)
    f = Field(stars=stars, masses=m, kappa_s=0.3, gamma=0.3,
              kappa_star=kappa_star, name="c3-clustered")
    f.grid = shooting_grid(0.5, 0.3, half_map, h, margin_frac=0.03, margin_min=5.0)
    f.box = (-half_map, half_map, -half_map, half_map)
    f.npx = f.npy = npix
    return f


def c4_critical(seed: int = 0, n: int = 200_000, npix: int = 8192,
                half_map: float = 1.0, h: float = 2.44e-4) -> Field:
    """Extremely magnified region near a critical curve: kappa_s=0.81,
    kappa_*=0.01, gamma=0.17 (mu ~ 286); masses uniform in [0.1, 1]."""
    f = config_uniform(seed, n, 0.01, 0.81, 0.17, mass_range=(0.1, 1.0),
                       name="c4-critical")
    f.grid = shooting_grid(0.82, 0.17, half_map, h, margin_frac=0.03,
                           margin_min=0.3)
    f.box = (-half_map, half_map, -half_map, half_map)
    f.npx = f.npy = npix
    return f


def nfw_halo(seed: int = 0, n: int = 10_000_000, q: float = 0.7,
             c: float = 10.0, r_s: float = 1.0, kappa_mean: float = 1.0,
             grid_n: int = 4096) -> Field:
    """Elliptical NFW halo of equal-mass particles: 3-D NFW (concentration c,
    truncated at c r_s) sampled by bisection on the enclosed-mass profile,
    projected, x2 squeezed by q; total mass set so the mean convergence over
    the +-2 r_s ray grid is ~kappa_mean.  Deflection-only workload."""
    rng = np.random.default_rng(seed)
    mu_of = lambda r: np.log1p(r) - r / (1.0 + r)
    target = rng.random(n) * mu_of(c)
    lo = np.zeros(n)
    hi = np.full(n, c)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = mu_of(mid) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    r = 0.5 * (lo + hi) * r_s
    cz = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    sz = np.sqrt(1.0 - cz * cz)
    stars = np.empty((n, 2))
    stars[:, 0] = r * sz * np.cos(ph)
    stars[:, 1] = q * r * sz * np.sin(ph)
    inside = (np.abs(stars[:, 0]) <= 2 * r_s) & (np.abs(stars[:, 1]) <= 2 * r_s)
    frac = max(float(np.mean(inside)), 1.0 / n)
    area = (4.0 * r_s) ** 2
    # kappa = pi * Sigma in Einstein units: pi * (M frac / area) = kappa_mean
    m_total = kappa_mean * area / (math.pi * frac)
    masses = np.full(n, m_total / n)
    f = Field(stars=stars, masses=masses, kappa_s=0.0, gamma=0.0,
              kappa_star=kappa_mean, name="nfw-halo")
    hh = 4.0 * r_s / grid_n
    f.grid = Grid(x0=-2.0 * r_s, y0=-2.0 * r_s, h=hh, nx=grid_n - 1, ny=grid_n - 1)
    return f


def c5_differentiable(seed: int = 0, n: int = 100_000, h: float = 0.01,
                      half_extent=(30.0, 2.5)) -> Field:
    """Differentiation workload: kappa_*=0.3, kappa_s=0.2, gamma=0.4, masses
    uniform in [0.5, 1.5]; rays over +-30 x +-2.5 ER at h=0.01."""
    f = config_uniform(seed, n, 0.3, 0.2, 0.4, mass_range=(0.5, 1.5),
                       name="c5-diff")
    nx = int(round(2 * half_extent[0] / h))
    ny = int(round(2 * half_extent[1] / h))
    f.grid = Grid(x0=-half_extent[0], y0=-half_extent[1], h=h, nx=nx, ny=ny)
    return f


def light_curve_track(n_samples: int = 2048, length: float = 5.0,
                      angle_deg: float = 30.0) -> np.ndarray:
    """Straight source track through the origin: (n_samples, 2)."""
    t = np.linspace(-0.5 * length, 0.5 * length, n_samples)
    a = math.radians(angle_deg)
    return np.stack([t * math.cos(a), t * math.sin(a)], axis=1)


def perturbed(field: Field, seed: int, sd: float = 0.01) -> Field:
    """Copy of a field with star positions jittered by N(0, sd^2) (seeded)."""
    rng = np.random.default_rng(seed)
    g = dataclasses.replace(field)
    g.stars = field.stars + rng.normal(0.0, sd, field.stars.shape)
    return g


def random_rays(seed: int, m: int, lo=(-1.0, -1.0), hi=(1.0, 1.0)) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = np.empty((m, 2))
    out[:, 0] = rng.uniform(lo[0], hi[0], m)
    out[:, 1] = rng.uniform(lo[1], hi[1], m)
    return out


def subsample_grid_rays(seed: int, grid: Grid, m: int) -> Tuple[np.ndarray, np.ndarray]:
    """m random corner rays of a grid: returns (indices (m, 2) as (i, j), positions (m, 2))."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, grid.nx + 1, m)
    j = rng.integers(0, grid.ny + 1, m)
    pos = np.stack([grid.x0 + i * grid.h, grid.y0 + j * grid.h], axis=1)
    return np.stack([i, j], axis=1), pos
