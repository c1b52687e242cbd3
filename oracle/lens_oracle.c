/*
 * lens_oracle.c -- plain, slow, FP64 CPU oracle for the FMM-IPM hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it (through oracle/__init__.py).  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Every routine is the plain definition written out, in the order and notation
 * of the paper (Jimenez-Vicente & Mediavilla 2022, "Fast Multipole Method for
 * Gravitational Lensing"):
 *
 *   oracle_deflect      -- Eq. 1 (lens equation, point lenses in Einstein
 *                          units) as an O(N* x N_x) direct sum (Sec. 2.1),
 *                          with the smooth convergence kappa_s and shear gamma
 *                          of the footnote to Eq. 1; optional analytic
 *                          Jacobian of the lens map.
 *   oracle_ipm_map      -- first-order Inverse Polygon Mapping (Sec. 2.3 and
 *                          the five-step FMM-IPM algorithm of Sec. 2.4): each
 *                          image-plane cell is mapped to a source-plane
 *                          quadrilateral and its area is apportioned to the
 *                          pixels it overlaps, mu = sum(S_i)/S*.
 *   oracle_ipm_map_refined -- the same with cells whose pixel box exceeds the
 *                          cap split into 2 x 2 sub-cells (new corner rays by
 *                          Eq. 1) up to a number of levels, instead of dropped
 *                          (the critical-cell refinement that the first-order
 *                          IPM of Sec. 2.3 leaves to a higher-order method).
 *   oracle_clip_area_sh -- polygon/pixel overlap by Sutherland-Hodgman
 *                          clipping + shoelace (used by oracle_ipm_map).
 *   oracle_clip_area_green -- the same overlap by an independent route: Green's
 *                          theorem edge integration (Sec. 2.3 names Green's
 *                          theorem as the apportioning rule).
 *   oracle_adjoint      -- gradient of a loss through Eq. 1 with respect to
 *                          star positions, masses, kappa_s and gamma, from the
 *                          real-variable derivatives of Eq. 1 (no complex
 *                          form, no FMM).
 *   oracle_multiplane_deflect -- rays through several thin lens planes (Sec.
 *                          1 and the footnote to the thin-lens approximation):
 *                          the multi-plane recursion, Eq. 1 at each plane.
 *   oracle_map_convolve_gaussian, oracle_histogram, oracle_map_track --
 *                          consumers of a map (Sec. 3): a Gaussian finite
 *                          source (direct 2D sum), magnification histograms,
 *                          light curves sampled along a source track.
 *   oracle_light_curve(_grad) -- light curve of a finite source (Sec. 3.3
 *                          derives light curves for Earendel; the source
 *                          profile is a Gaussian, as for the background source
 *                          of Sec. 2.5) written as a ray sum, and its
 *                          derivative with respect to the mapped rays.
 *
 * Readings of points the paper leaves open (all also used by the CUDA path,
 * which implements them independently):
 *   - smooth field: y1 = (1-kappa_s-gamma) x1 - alpha1,
 *                   y2 = (1-kappa_s+gamma) x2 - alpha2  (shear along x1);
 *   - a star exactly at a ray contributes nothing (self-interaction skipped);
 *   - IPM: signed-area fraction a_pix / A_P of the mapped cell; cells with
 *     |A_P| <= 1e-14 * A_cell are "degenerate" and skipped; cells whose pixel
 *     bounding box lies entirely outside the map go to "outside"; cells whose
 *     pixel bounding box spans more than bbox_cap pixels on a side (cap > 0)
 *     are "dropped"; every category is booked in a flux ledger;
 *   - finite source (Sec. 3 histograms of sources of given size): a circular
 *     Gaussian profile of sigma pixels cut at the isophote |d| = trunc sigma,
 *     renormalised to its part inside the map.
 *
 * Parity pins for every routine live in tests/test_oracle_*.py.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Threads the OpenMP loops of this file use (reported with the timings of
 * the CPU baseline). */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Neumaier-compensated running sum (so the oracle itself is ~1e-15 exact). */
typedef struct { double s, c; } nsum;
static inline void nsum_add(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static inline double nsum_get(const nsum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Eq. 1: y = x - sum_i m_i (x - x_i)/|x - x_i|^2, plus the smooth field.
 * stars: n x 2 (x1, x2) interleaved; masses: n; rays: m x 2.
 * y_out: m x 2.  alpha_out (m x 2) and jac_out (m x 4, row-major dy/dx:
 * [dy1/dx1, dy1/dx2, dy2/dx1, dy2/dx2]) are optional (NULL to skip). */
void oracle_deflect(int64_t n, const double* stars, const double* masses,
                    double kappa_s, double gamma, int64_t m, const double* rays,
                    double* y_out, double* alpha_out, double* jac_out) {
  const double a = 1.0 - kappa_s - gamma;
  const double b = 1.0 - kappa_s + gamma;
  /* one ray per scheduling unit: with a million stars a ray is milliseconds
   * of work, and small samples still spread over every core */
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < m; ++r) {
    const double x1 = rays[2 * r], x2 = rays[2 * r + 1];
    nsum s1 = {0, 0}, s2 = {0, 0};
    nsum j11 = {0, 0}, j12 = {0, 0}, j22 = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
      const double d1 = x1 - stars[2 * i];
      const double d2 = x2 - stars[2 * i + 1];
      const double r2 = d1 * d1 + d2 * d2;
      if (r2 == 0.0) continue; /* self-interaction skipped */
      const double w = masses[i] / r2;
      nsum_add(&s1, w * d1);
      nsum_add(&s2, w * d2);
      if (jac_out) {
        /* d alpha / d x of m d/|d|^2 = m (I |d|^2 - 2 d d^T)/|d|^4 */
        const double w2 = w / r2;
        nsum_add(&j11, w2 * (d2 * d2 - d1 * d1));
        nsum_add(&j12, w2 * (-2.0 * d1 * d2));
        nsum_add(&j22, w2 * (d1 * d1 - d2 * d2));
      }
    }
    const double al1 = nsum_get(&s1), al2 = nsum_get(&s2);
    y_out[2 * r] = a * x1 - al1;
    y_out[2 * r + 1] = b * x2 - al2;
    if (alpha_out) {
      alpha_out[2 * r] = al1;
      alpha_out[2 * r + 1] = al2;
    }
    if (jac_out) {
      const double da11 = nsum_get(&j11), da12 = nsum_get(&j12), da22 = nsum_get(&j22);
      jac_out[4 * r + 0] = a - da11;
      jac_out[4 * r + 1] = -da12;
      jac_out[4 * r + 2] = -da12;
      jac_out[4 * r + 3] = b - da22;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Polygon / axis-aligned-square overlap, route 1: Sutherland-Hodgman.
 * Clipping against a convex window keeps the winding-number-weighted area of
 * any closed polygon (self-intersecting or inverted included), so the signed
 * shoelace area of the clipped polygon is the signed overlap. */
#define SH_MAXV 256
static int sh_clip_half(const double* in, int nin, double* out, int axis,
                        double bound, int keep_ge) {
  int nout = 0;
  if (nin == 0) return 0;
  for (int k = 0; k < nin; ++k) {
    const double* P = in + 2 * k;
    const double* Q = in + 2 * ((k + 1) % nin);
    const double pv = P[axis] - bound, qv = Q[axis] - bound;
    const int pin = keep_ge ? (pv >= 0) : (pv <= 0);
    const int qin = keep_ge ? (qv >= 0) : (qv <= 0);
    if (pin) {
      out[2 * nout] = P[0]; out[2 * nout + 1] = P[1]; ++nout;
    }
    if (pin != qin) {
      const double t = pv / (pv - qv);
      double X[2];
      X[0] = P[0] + t * (Q[0] - P[0]);
      X[1] = P[1] + t * (Q[1] - P[1]);
      X[axis] = bound;
      out[2 * nout] = X[0]; out[2 * nout + 1] = X[1]; ++nout;
    }
  }
  return nout;
}

/* Signed (counter-clockwise positive) area, taken about the first vertex so
 * that far-from-origin polygons keep their digits. */
static double shoelace(const double* v, int n) {
  double s = 0.0;
  const double ox = v[0], oy = v[1];
  for (int k = 1; k + 1 < n; ++k) {
    const double px = v[2 * k] - ox, py = v[2 * k + 1] - oy;
    const double qx = v[2 * k + 2] - ox, qy = v[2 * k + 3] - oy;
    s += px * qy - qx * py;
  }
  return 0.5 * s;
}

/* Signed area of polygon (n vertices, interleaved x,y) inside the square
 * [x0, x0+1] x [y0, y0+1]. */
double oracle_clip_area_sh(const double* poly, int n, double x0, double y0) {
  double A[2 * SH_MAXV], B[2 * SH_MAXV];
  if (n > 16) return NAN;
  memcpy(A, poly, sizeof(double) * 2 * n);
  int k = n;
  k = sh_clip_half(A, k, B, 0, x0, 1);
  k = sh_clip_half(B, k, A, 0, x0 + 1.0, 0);
  k = sh_clip_half(A, k, B, 1, y0, 1);
  k = sh_clip_half(B, k, A, 1, y0 + 1.0, 0);
  if (k < 3) return 0.0;
  return shoelace(A, k);
}

/* Route 2: Green's theorem.  With g(x, y) = clamp(x, x0, x1) - x0 on the strip
 * y0 <= y <= y1 (and 0 off it) we have dg/dx = indicator of the square, so
 * the winding-weighted overlap is the contour integral of g dy along the
 * polygon.  Each edge is a straight segment; on it g is piecewise linear in
 * the edge parameter, so integrating piece by piece (split where x crosses
 * x0 or x1) is exact. */
static double edge_integral(double xa, double ya, double xb, double yb,
                            double x0, double x1, double y0, double y1) {
  if (ya == yb) return 0.0; /* dy = 0 along the edge */
  /* parameter interval where y is inside [y0, y1] */
  double t0 = (y0 - ya) / (yb - ya), t1 = (y1 - ya) / (yb - ya);
  if (t0 > t1) { double tt = t0; t0 = t1; t1 = tt; }
  if (t0 < 0.0) t0 = 0.0;
  if (t1 > 1.0) t1 = 1.0;
  if (t0 >= t1) return 0.0;
  /* break points where x crosses x0 or x1 */
  double ts[4];
  int nt = 0;
  ts[nt++] = t0;
  if (xb != xa) {
    double c0 = (x0 - xa) / (xb - xa), c1 = (x1 - xa) / (xb - xa);
    if (c0 > c1) { double tt = c0; c0 = c1; c1 = tt; }
    if (c0 > t0 && c0 < t1) ts[nt++] = c0;
    if (c1 > t0 && c1 < t1) ts[nt++] = c1;
  }
  ts[nt++] = t1;
  double sum = 0.0;
  for (int k = 0; k + 1 < nt; ++k) {
    const double ta = ts[k], tb = ts[k + 1];
    /* g is linear on [ta, tb]; the trapezoid rule with the clamped end
     * values is exact unless a clamp kink sits inside, which the split
     * excludes.  Evaluate g at both ends. */
    double xa_ = xa + ta * (xb - xa), xb_ = xa + tb * (xb - xa);
    double ga = (xa_ < x0 ? x0 : (xa_ > x1 ? x1 : xa_)) - x0;
    double gb = (xb_ < x0 ? x0 : (xb_ > x1 ? x1 : xb_)) - x0;
    const double dy = (tb - ta) * (yb - ya);
    sum += 0.5 * (ga + gb) * dy;
  }
  return sum;
}

double oracle_clip_area_green(const double* poly, int n, double x0, double y0) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    const double* P = poly + 2 * k;
    const double* Q = poly + 2 * ((k + 1) % n);
    s += edge_integral(P[0], P[1], Q[0], Q[1], x0, x0 + 1.0, y0, y0 + 1.0);
  }
  return s;
}

/* ------------------------------------------------------------------------ */
/* First-order IPM (Sec. 2.3): cells of the image-plane grid are mapped with
 * the lens equation; each mapped quadrilateral's area is apportioned to the
 * source-plane pixels it overlaps.  The cell (i, j) has corners
 *   y[j][i], y[j][i+1], y[j+1][i+1], y[j+1][i]
 * (counter-clockwise in the image plane), taken from ycorn, a row-major
 * (ny+1) x (nx+1) x 2 array.  h is the cell side (A_cell = h^2).  The map
 * covers [u0, u1) x [v0, v1) in source-plane coordinates with npx x npy
 * pixels; pixel (px, py) is map[py * npx + px].  On return
 *   map[pix] = sum_cells A_cell * a_pix / A_P / S*     (S* = pixel area)
 * i.e. the magnification mu = sum S_i / S*.
 * stats (8 doubles): [0] cells, [1] area_total, [2] area_in_map,
 *   [3] area_outside, [4] area_dropped, [5] area_degenerate,
 *   [6] cells_dropped, [7] cells_degenerate. */
/* The state one IPM pass accumulates into. */
typedef struct {
  double u0, v0, du, dv, S_star;
  int npx, npy, bbox_cap;
  double* map;
  nsum in_map, outside, dropped, degen;
  double n_dropped, n_degen;
  /* refinement: the lens, the grid origin, the levels allowed */
  int64_t n;
  const double *stars, *masses;
  double kappa_s, gamma;
  int levels;
} ipm_ctx;

/* One (sub)cell of side hc whose deflected corners are P (c00, c10, c11,
 * c01), lower-left image-plane corner (xl, yl), at refinement level `level`. */
static void ipm_cell(ipm_ctx* c, const double P[8], double xl, double yl, double hc, int level) {
  const double A_cell = hc * hc;
  /* source-plane area of the mapped cell */
  const double A_P = shoelace(P, 4);
  if (!(fabs(A_P) > 1e-14 * A_cell)) {
    nsum_add(&c->degen, A_cell); c->n_degen += 1; return;
  }
  /* pixel coordinates */
  double Q[8];
  for (int k = 0; k < 4; ++k) {
    Q[2 * k] = (P[2 * k] - c->u0) / c->du;
    Q[2 * k + 1] = (P[2 * k + 1] - c->v0) / c->dv;
  }
  double qmin0 = Q[0], qmax0 = Q[0], qmin1 = Q[1], qmax1 = Q[1];
  for (int k = 1; k < 4; ++k) {
    qmin0 = fmin(qmin0, Q[2 * k]); qmax0 = fmax(qmax0, Q[2 * k]);
    qmin1 = fmin(qmin1, Q[2 * k + 1]); qmax1 = fmax(qmax1, Q[2 * k + 1]);
  }
  const double fx0 = floor(qmin0), fx1 = floor(qmax0);
  const double fy0 = floor(qmin1), fy1 = floor(qmax1);
  const int npx = c->npx, npy = c->npy;
  if (fx1 < 0 || fy1 < 0 || fx0 > npx - 1 || fy0 > npy - 1) {
    nsum_add(&c->outside, A_cell); return;
  }
  if (c->bbox_cap > 0 && (fx1 - fx0 + 1 > c->bbox_cap || fy1 - fy0 + 1 > c->bbox_cap)) {
    if (level < c->levels) {
      /* 2 x 2 sub-cells of half the side: the five new corner rays (edge
       * midpoints and centre) through the lens equation */
      const double g = 0.5 * hc;
      const double X[10] = {xl + g, yl, xl + hc, yl + g, xl + g, yl + hc, xl, yl + g, xl + g, yl + g};
      double Y[10];
      oracle_deflect(c->n, c->stars, c->masses, c->kappa_s, c->gamma, 5, X, Y, NULL, NULL);
      /* 3 x 3 corner grid G[row][col], rows along x2 */
      const double* G[3][3] = {{P + 0, Y + 0, P + 2}, {Y + 6, Y + 8, Y + 2}, {P + 6, Y + 4, P + 4}};
      for (int bq = 0; bq < 2; ++bq)
        for (int aq = 0; aq < 2; ++aq) {
          const double* k00 = G[bq][aq];
          const double* k10 = G[bq][aq + 1];
          const double* k11 = G[bq + 1][aq + 1];
          const double* k01 = G[bq + 1][aq];
          const double S[8] = {k00[0], k00[1], k10[0], k10[1], k11[0], k11[1], k01[0], k01[1]};
          ipm_cell(c, S, xl + aq * g, yl + bq * g, g, level + 1);
        }
      return;
    }
    nsum_add(&c->dropped, A_cell); c->n_dropped += 1; return;
  }
  const double A_Pp = A_P / c->S_star; /* area in pixel units */
  const int64_t ix0 = fx0 < 0 ? 0 : (int64_t)fx0;
  const int64_t ix1 = fx1 > npx - 1 ? npx - 1 : (int64_t)fx1;
  const int64_t iy0 = fy0 < 0 ? 0 : (int64_t)fy0;
  const int64_t iy1 = fy1 > npy - 1 ? npy - 1 : (int64_t)fy1;
  double frac_in = 0.0;
  for (int64_t py = iy0; py <= iy1; ++py) {
    for (int64_t px = ix0; px <= ix1; ++px) {
      const double a = oracle_clip_area_sh(Q, 4, (double)px, (double)py);
      if (a == 0.0) continue;
      const double frac = a / A_Pp;
      c->map[py * npx + px] += A_cell * frac;
      frac_in += frac;
    }
  }
  nsum_add(&c->in_map, A_cell * frac_in);
  nsum_add(&c->outside, A_cell * (1.0 - frac_in));
}

static void ipm_run(ipm_ctx* c, int64_t nx, int64_t ny, double x0, double y0, double h,
                    const double* ycorn, double* stats) {
  const int64_t W = nx + 1;
  for (int64_t p = 0; p < (int64_t)c->npx * c->npy; ++p) c->map[p] = 0.0;
  for (int64_t j = 0; j < ny; ++j) {
    for (int64_t i = 0; i < nx; ++i) {
      const double* c00 = ycorn + 2 * (j * W + i);
      const double* c10 = ycorn + 2 * (j * W + i + 1);
      const double* c11 = ycorn + 2 * ((j + 1) * W + i + 1);
      const double* c01 = ycorn + 2 * ((j + 1) * W + i);
      const double P[8] = {c00[0], c00[1], c10[0], c10[1], c11[0], c11[1], c01[0], c01[1]};
      ipm_cell(c, P, x0 + (double)i * h, y0 + (double)j * h, h, 0);
    }
  }
  for (int64_t p = 0; p < (int64_t)c->npx * c->npy; ++p) c->map[p] /= c->S_star;
  stats[0] = (double)nx * (double)ny;
  stats[1] = stats[0] * h * h;
  stats[2] = nsum_get(&c->in_map);
  stats[3] = nsum_get(&c->outside);
  stats[4] = nsum_get(&c->dropped);
  stats[5] = nsum_get(&c->degen);
  stats[6] = c->n_dropped;
  stats[7] = c->n_degen;
}

void oracle_ipm_map(int64_t nx, int64_t ny, double h, const double* ycorn,
                    double u0, double u1, double v0, double v1, int npx, int npy,
                    int bbox_cap, double* map, double* stats) {
  ipm_ctx c;
  memset(&c, 0, sizeof(c));
  c.u0 = u0; c.v0 = v0;
  c.du = (u1 - u0) / npx; c.dv = (v1 - v0) / npy;
  c.S_star = c.du * c.dv;
  c.npx = npx; c.npy = npy; c.bbox_cap = bbox_cap;
  c.map = map;
  ipm_run(&c, nx, ny, 0.0, 0.0, h, ycorn, stats);
}

/* Refined IPM: as oracle_ipm_map, but a cell whose pixel box spans more
 * than bbox_cap pixels on a side is split into 2 x 2 sub-cells of half the
 * side, the five new corner rays deflected by Eq. 1 (direct sum), up to
 * `levels` times; a sub-cell still too large at the last level is dropped.
 * The grid's cell (i, j) has its lower-left corner at (x0 + i h, y0 + j h)
 * and ycorn holds the deflected corners of the grid.  levels = 0 gives
 * oracle_ipm_map. */
void oracle_ipm_map_refined(int64_t nx, int64_t ny, double x0, double y0, double h,
                            const double* ycorn, int64_t n, const double* stars,
                            const double* masses, double kappa_s, double gamma, double u0,
                            double u1, double v0, double v1, int npx, int npy, int bbox_cap,
                            int levels, double* map, double* stats) {
  ipm_ctx c;
  memset(&c, 0, sizeof(c));
  c.u0 = u0; c.v0 = v0;
  c.du = (u1 - u0) / npx; c.dv = (v1 - v0) / npy;
  c.S_star = c.du * c.dv;
  c.npx = npx; c.npy = npy; c.bbox_cap = bbox_cap;
  c.map = map;
  c.n = n; c.stars = stars; c.masses = masses; c.kappa_s = kappa_s; c.gamma = gamma;
  c.levels = levels;
  ipm_run(&c, nx, ny, x0, y0, h, ycorn, stats);
}

/* ------------------------------------------------------------------------ */
/* Gradient of a loss L(y) through Eq. 1 (real-variable form).
 * gy: m x 2 = dL/dy at every ray.  With d = x_r - x_j and
 *   alpha_r = sum_j m_j d / |d|^2,   y_r = diag(a, b) x_r - alpha_r,
 * dL/dalpha_r = -gy_r, so
 *   dL/dm_j   = sum_r (-gy_r) . d / |d|^2
 *   dL/dx_j   = sum_r (-gy_r)^T d alpha_r / d x_j
 *             = m_j sum_r J(d)^T gy_r,  J(d) = (I |d|^2 - 2 d d^T)/|d|^4
 *   dL/dkappa_s = -sum_r (gy1 x1 + gy2 x2)
 *   dL/dgamma   = sum_r (-gy1 x1 + gy2 x2)
 * Outputs: gxy (n x 2), gm (n), gkg (2). */
void oracle_adjoint(int64_t n, const double* stars, const double* masses,
                    int64_t m, const double* rays, const double* gy,
                    double* gxy, double* gm, double* gkg) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t j = 0; j < n; ++j) {
    const double xj1 = stars[2 * j], xj2 = stars[2 * j + 1], mj = masses[j];
    nsum s_m = {0, 0}, s_1 = {0, 0}, s_2 = {0, 0};
    for (int64_t r = 0; r < m; ++r) {
      const double d1 = rays[2 * r] - xj1, d2 = rays[2 * r + 1] - xj2;
      const double r2 = d1 * d1 + d2 * d2;
      if (r2 == 0.0) continue;
      const double g1 = gy[2 * r], g2 = gy[2 * r + 1];
      nsum_add(&s_m, -(g1 * d1 + g2 * d2) / r2);
      const double r4 = r2 * r2;
      const double J11 = (r2 - 2.0 * d1 * d1) / r4;
      const double J12 = (-2.0 * d1 * d2) / r4;
      const double J22 = (r2 - 2.0 * d2 * d2) / r4;
      nsum_add(&s_1, J11 * g1 + J12 * g2);
      nsum_add(&s_2, J12 * g1 + J22 * g2);
    }
    gm[j] = nsum_get(&s_m);
    gxy[2 * j] = mj * nsum_get(&s_1);
    gxy[2 * j + 1] = mj * nsum_get(&s_2);
  }
  nsum sk = {0, 0}, sg = {0, 0};
  for (int64_t r = 0; r < m; ++r) {
    const double x1 = rays[2 * r], x2 = rays[2 * r + 1];
    const double g1 = gy[2 * r], g2 = gy[2 * r + 1];
    nsum_add(&sk, -(g1 * x1 + g2 * x2));
    nsum_add(&sg, -g1 * x1 + g2 * x2);
  }
  gkg[0] = nsum_get(&sk);
  gkg[1] = nsum_get(&sg);
}

/* ------------------------------------------------------------------------ */
/* Light curve of a circular Gaussian source of width sigma moving through
 * the samples s_k (ns x 2) of the source plane: every ray carries the
 * image-plane area w_ray, so
 *   F_k = sum_r w_ray exp(-|y_r - s_k|^2 / (2 sigma^2)) / (2 pi sigma^2),
 * the source's magnification at s_k.  Pairs farther than trunc*sigma are
 * left out (both sides of the parity test use the same cut). */
void oracle_light_curve(int64_t m, const double* y, double w_ray, int64_t ns,
                        const double* s, double sigma, double trunc, double* F) {
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  const double norm = w_ray / (2.0 * M_PI * sigma * sigma);
  const double cut2 = trunc * trunc * sigma * sigma;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < ns; ++k) {
    nsum acc = {0, 0};
    for (int64_t r = 0; r < m; ++r) {
      const double d1 = y[2 * r] - s[2 * k], d2 = y[2 * r + 1] - s[2 * k + 1];
      const double q = d1 * d1 + d2 * d2;
      if (q > cut2) continue;
      nsum_add(&acc, exp(-q * inv2s2));
    }
    F[k] = norm * nsum_get(&acc);
  }
}

/* dL/dy for L = sum_k (F_k - T_k)^2, given F (from oracle_light_curve). */
void oracle_light_curve_grad(int64_t m, const double* y, double w_ray, int64_t ns,
                             const double* s, double sigma, double trunc,
                             const double* F, const double* T, double* gy) {
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  const double norm = w_ray / (2.0 * M_PI * sigma * sigma);
  const double cut2 = trunc * trunc * sigma * sigma;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t r = 0; r < m; ++r) {
    nsum g1 = {0, 0}, g2 = {0, 0};
    for (int64_t k = 0; k < ns; ++k) {
      const double d1 = y[2 * r] - s[2 * k], d2 = y[2 * r + 1] - s[2 * k + 1];
      const double q = d1 * d1 + d2 * d2;
      if (q > cut2) continue;
      /* d/dy of exp(-q/(2 s^2)) = -exp(.) * d / s^2 */
      const double e = 2.0 * (F[k] - T[k]) * norm * exp(-q * inv2s2) * (-2.0 * inv2s2);
      nsum_add(&g1, e * d1);
      nsum_add(&g2, e * d2);
    }
    gy[2 * r] = nsum_get(&g1);
    gy[2 * r + 1] = nsum_get(&g2);
  }
}

/* ------------------------------------------------------------------------ */
/* Several thin lens planes (Sec. 1: thick lenses and cosmological ray tracing
 * take several lens planes, the mapping repeated plane by plane; footnote to
 * the thin-lens approximation: a 3D lens as a collection of thin planes).
 * K planes in order of distance from the observer; plane i holds n[i] point
 * lenses (stars[i]: n[i] x 2, masses[i]: n[i]) and a smooth field (kappa[i],
 * gamma[i]), each deflection scaled to the source plane as in Eq. 1:
 *   alpha_i(x) = sum_k m_ik (x - x_ik) / |x - x_ik|^2
 *                + diag(kappa_i + gamma_i, kappa_i - gamma_i) x.
 * A ray enters plane 1 at x_1 = x, reaches plane j at
 *   x_j = x_1 - sum_{i<j} beta[i K + j] alpha_i(x_i)      (j = 2 .. K)
 * and the source plane at
 *   y = x_1 - sum_{i<=K} alpha_i(x_i),
 * beta[i K + j] (i < j, 0-based) being the distance ratio D_ij D_s / (D_j D_is)
 * of the pair (entries with i >= j are not read).  With K = 1 this is Eq. 1.
 * y_out: m x 2; xplanes_out: K x m x 2 (x_i per plane) or NULL. */
void oracle_multiplane_deflect(int K, const int64_t* n, const double* const* stars,
                               const double* const* masses, const double* kappa,
                               const double* gamma, const double* beta, int64_t m,
                               const double* rays, double* y_out, double* xplanes_out) {
  double* x = (double*)malloc(sizeof(double) * 2 * (size_t)(m > 0 ? m : 1));
  double* al = (double*)malloc(sizeof(double) * 2 * (size_t)(m > 0 ? m : 1));
  double* yt = (double*)malloc(sizeof(double) * 2 * (size_t)(m > 0 ? m : 1));
  /* sum over the planes seen so far of beta_ij alpha_i, for every later plane j
   * (acc[j] for j < K) and for the source plane (acc[K], beta = 1) */
  double* acc = (double*)calloc((size_t)(K + 1) * 2 * (size_t)(m > 0 ? m : 1), sizeof(double));
  for (int i = 0; i < K; ++i) {
    /* x_i = x_1 - (sum of the earlier planes' deflections weighted for plane i) */
    for (int64_t r = 0; r < 2 * m; ++r) x[r] = rays[r] - acc[(size_t)i * 2 * m + r];
    if (xplanes_out)
      for (int64_t r = 0; r < 2 * m; ++r) xplanes_out[(size_t)i * 2 * m + r] = x[r];
    if (n[i] > 0) {
      oracle_deflect(n[i], stars[i], masses[i], 0.0, 0.0, m, x, yt, al, NULL);
    } else {
      for (int64_t r = 0; r < 2 * m; ++r) al[r] = 0.0;
    }
    for (int64_t r = 0; r < m; ++r) {
      al[2 * r] += (kappa[i] + gamma[i]) * x[2 * r];
      al[2 * r + 1] += (kappa[i] - gamma[i]) * x[2 * r + 1];
    }
    for (int j = i + 1; j <= K; ++j) {
      const double bij = j < K ? beta[(size_t)i * K + j] : 1.0;
      double* aj = acc + (size_t)j * 2 * m;
      for (int64_t r = 0; r < 2 * m; ++r) aj[r] += bij * al[r];
    }
  }
  for (int64_t r = 0; r < 2 * m; ++r) y_out[r] = rays[r] - acc[(size_t)K * 2 * m + r];
  free(x);
  free(al);
  free(yt);
  free(acc);
}

/* ------------------------------------------------------------------------ */
/* Consumers of a magnification map (Sec. 3: histograms of the magnification
 * of finite sources, light curves along source tracks).  The map is npy x npx,
 * row-major, pixel (px, py) centred at (px + 1/2, py + 1/2) in pixel units.
 *
 * Finite source: the map seen by a circular Gaussian source of sigma_px
 * pixels, the source's profile cut at the isophote |d| = trunc sigma (where
 * its brightness has fallen to exp(-trunc^2 / 2) of the peak) and
 * renormalised to the part of the profile that lies inside the map:
 *   out[p] = sum_q w(q - p) map[q] / sum_q w(q - p),  w(d) = exp(-|d|^2 / 2 s^2),
 * q over the map pixels with |q - p|^2 <= (trunc s)^2.  Plain 2D sum. */
void oracle_map_convolve_gaussian(int npx, int npy, const double* map, double sigma_px,
                                  double trunc, double* out) {
  const int R = (int)floor(trunc * sigma_px);
  const double inv2s2 = 1.0 / (2.0 * sigma_px * sigma_px);
  const double cut2 = trunc * trunc * sigma_px * sigma_px;
#pragma omp parallel for schedule(dynamic, 4)
  for (int py = 0; py < npy; ++py) {
    for (int px = 0; px < npx; ++px) {
      nsum num = {0, 0}, den = {0, 0};
      for (int dy = -R; dy <= R; ++dy) {
        const int qy = py + dy;
        if (qy < 0 || qy >= npy) continue;
        for (int dx = -R; dx <= R; ++dx) {
          const int qx = px + dx;
          if (qx < 0 || qx >= npx) continue;
          const double d2 = (double)dx * dx + (double)dy * dy;
          if (d2 > cut2) continue;
          const double w = exp(-d2 * inv2s2);
          nsum_add(&num, w * map[(int64_t)qy * npx + qx]);
          nsum_add(&den, w);
        }
      }
      out[(int64_t)py * npx + px] = nsum_get(&num) / nsum_get(&den);
    }
  }
}

/* Histogram of n values into nbins equal bins of [lo, hi) (of log10(value)
 * when log_bins, values <= 0 counting as below): counts[0] below lo,
 * counts[1 .. nbins] the bins, counts[nbins + 1] at or above hi. */
void oracle_histogram(int64_t n, const double* v, double lo, double hi, int nbins, int log_bins,
                      int64_t* counts) {
  for (int b = 0; b < nbins + 2; ++b) counts[b] = 0;
  for (int64_t i = 0; i < n; ++i) {
    double x = v[i];
    if (log_bins) {
      if (!(x > 0.0)) { counts[0] += 1; continue; }
      x = log10(x);
    }
    if (x < lo) { counts[0] += 1; continue; }
    if (x >= hi) { counts[nbins + 1] += 1; continue; }
    int b = (int)floor((x - lo) / (hi - lo) * nbins);
    if (b >= nbins) b = nbins - 1;
    counts[1 + b] += 1;
  }
}

/* The map at ns source positions s (source-plane coordinates, the map
 * covering [u0, u1) x [v0, v1)), bilinear between pixel centres, clamped to
 * the outermost centres: a light curve along a track of the source. */
void oracle_map_track(int npx, int npy, const double* map, double u0, double u1, double v0,
                      double v1, int64_t ns, const double* s, double* out) {
  const double du = (u1 - u0) / npx, dv = (v1 - v0) / npy;
  for (int64_t k = 0; k < ns; ++k) {
    double x = (s[2 * k] - u0) / du - 0.5, y = (s[2 * k + 1] - v0) / dv - 0.5;
    x = fmin(fmax(x, 0.0), (double)(npx - 1));
    y = fmin(fmax(y, 0.0), (double)(npy - 1));
    int ix = (int)floor(x), iy = (int)floor(y);
    if (ix > npx - 2) ix = npx > 1 ? npx - 2 : 0;
    if (iy > npy - 2) iy = npy > 1 ? npy - 2 : 0;
    const double fx = npx > 1 ? x - ix : 0.0, fy = npy > 1 ? y - iy : 0.0;
    const int ix1 = npx > 1 ? ix + 1 : ix, iy1 = npy > 1 ? iy + 1 : iy;
    const double m00 = map[(int64_t)iy * npx + ix], m10 = map[(int64_t)iy * npx + ix1];
    const double m01 = map[(int64_t)iy1 * npx + ix], m11 = map[(int64_t)iy1 * npx + ix1];
    out[k] = (1 - fy) * ((1 - fx) * m00 + fx * m10) + fy * ((1 - fx) * m01 + fx * m11);
  }
}
