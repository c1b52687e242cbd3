// lightcurve.cu -- Gaussian-source light curve as a ray sum and its gradient
// with respect to the mapped rays.  A source of profile
// G(s) = exp(-|s|^2 / (2 sigma^2)) / (2 pi sigma^2) (the Gaussian source of
// Sec. 2.5) centred at s_k has magnification F_k = sum_r w_ray G(y_r - s_k)
// when every ray carries the image-plane area w_ray; sampling s_k along a
// track gives a light curve (Sec. 3.3).  Pairs with |y_r - s_k| > trunc sigma
// are left out.  L = sum_k (F_k - T_k)^2 gives
//   dL/dy_r = sum_k 2 (F_k - T_k) w_ray G(y_r - s_k) (-(y_r - s_k) / sigma^2).
// Samples are bucketed on a uniform grid of cell >= trunc*sigma.  The forward
// pass buckets the rays near the samples on the same grid (one cell wider)
// and gives each sample a block that sums over the rays of the 3 x 3 cells
// around it (no atomics); the gradient gives each ray a thread that sums over
// the samples of the 3 x 3 cells around it, the samples stored in cell order
// with their coefficients.  A pair's difference, cut test, Gaussian and sums
// are float-float (pairs of float32, ~48 bits) on the float32 pipe -- GB300's
// float64 pipe is 1/74 of float32 -- and a plain float32 test with a margin
// for its rounding skips the pairs clearly beyond the cut.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kLcThreads = 256;

// exp(x), x <= 0, in float-float by the table-driven method of Tang ("Table-
// driven implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989): x = (64 m + j) ln2/64 + r with
// |r| <= ln2/128, exp(x) = 2^m 2^(j/64) exp(r); 2^(j/64) from a float-float
// table, exp(r) from its Taylor series, 1 + r + r^2/2 in float-float and the
// terms from r^3/6 (< 3e-8) on in float32.  ln2/64 is split as L1 + L2 + L3,
// L1 with 11 significant bits, so that k L1 is exact for |k| < 2^13.  Below
// x = -87 (2^m under the float32 normal range) the result is 0.
struct ExpTab {
  float thi[64], tlo[64];  // 2^(j/64)
  float l1, l2, l3;        // ln2/64
};

ExpTab make_exp_tab() {
  ExpTab t{};
  for (int j = 0; j < 64; ++j) {
    const double v = std::exp2(j / 64.0);
    t.thi[j] = (float)v;
    t.tlo[j] = (float)(v - (double)t.thi[j]);
  }
  const double L = std::log(2.0) / 64.0;
  const double l1 = std::ldexp(std::nearbyint(std::ldexp(L, 17)), -17);  // 11 bits
  t.l1 = (float)l1;
  t.l2 = (float)(L - l1);
  t.l3 = (float)(L - l1 - (double)t.l2);
  return t;
}

__device__ __forceinline__ ff ff_exp_neg(ff x, const ExpTab& T) {
  if (!(x.hi > -87.0f)) return ff{0.f, 0.f};
  const float kf = rintf(x.hi * 92.33248261689366f);  // 64 / ln2
  const int k = (int)kf;
  const int m = k >> 6, j = k - (m << 6);
  // r = x - k ln2/64: x.hi - k L1 is exact (Sterbenz), -k L2 an exact product
  const float a = fmaf(-kf, T.l1, x.hi);
  const float p = -kf * T.l2;
  const float pe = fmaf(-kf, T.l2, -p);
  float s, e;
  two_sum(a, p, s, e);
  e += pe + x.lo - kf * T.l3;
  const ff r = ff_norm(s, e);
  // 1 + r + r^2/2 + r^3/6 + ... + r^6/720
  const float r2h = r.hi * r.hi;
  const float r2l = fmaf(r.hi, r.hi, -r2h) + 2.f * r.hi * r.lo;
  const float tail =
      r2h * r.hi * fmaf(r.hi, fmaf(r.hi, fmaf(r.hi, 1.f / 720.f, 1.f / 120.f), 1.f / 24.f), 1.f / 6.f);
  ff E = ff_add(ff{1.f, 0.f}, r);
  E = ff_add(E, ff_norm(0.5f * r2h, 0.5f * r2l));
  E = ff_add(E, tail);
  E = ff_mul(E, ff{T.thi[j], T.tlo[j]});
  const float sc = __int_as_float((127 + m) << 23);  // 2^m, m >= -126
  return ff{E.hi * sc, E.lo * sc};
}

__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// Positions are kept as a cell of the sample grid (a side of three significant
// bits, origin a multiple of it) and the offset from that cell's origin, exact in float64
// (|offset| < 2 cells) and then float-float: the difference of two points is
// (a - b) + (cell_a - cell_b) * side, to ~2^-48 of a cell whatever the
// coordinates' size.
struct Pos {
  float4 o;  // offset: x hi, x lo, y hi, y lo
  int2 c;    // cell
};
__device__ __forceinline__ Pos make_pos(double x, double y, int cx, int cy, double x0, double y0,
                                        double side) {
  const ff a = ff_of(x - (x0 + cx * side)), b = ff_of(y - (y0 + cy * side));
  return Pos{make_float4(a.hi, a.lo, b.hi, b.lo), make_int2(cx, cy)};
}

// The Gaussian of a pair, G = exp(-|d|^2 / (2 sigma^2)) with d = y - s, in
// float-float; false beyond the cut (q = |d|^2 > cut2).  A float32 test
// first: the offsets' hi parts are within 2^-24 of 2 cells of the truth and
// the cell term is exact, so a margin of 2^-21 cells covers their rounding
// and that of d and q; it rejects only pairs surely beyond the cut.
__device__ __forceinline__ bool pair_gauss(const Pos& y, const Pos& s, float side, float cutf,
                                           ff ninv2s2, ff cut2, const ExpTab& T, ff& d1, ff& d2,
                                           ff& G) {
  const float cx = (float)(y.c.x - s.c.x) * side, cy = (float)(y.c.y - s.c.y) * side;
  const float e1 = (y.o.x - s.o.x) + cx, e2 = (y.o.z - s.o.z) + cy;
  const float c = cutf * 1.00001f + 4.8e-7f * side;
  if (fmaf(e1, e1, e2 * e2) > c * c) return false;
  d1 = ff_add(ff_add(ff{y.o.x, y.o.y}, ff{-s.o.x, -s.o.y}), cx);
  d2 = ff_add(ff_add(ff{y.o.z, y.o.w}, ff{-s.o.z, -s.o.w}), cy);
  const ff q = ff_add(ff_mul(d1, d1), ff_mul(d2, d2));
  if (ff_gt(q, cut2)) return false;
  G = ff_exp_neg(ff_mul(q, ninv2s2), T);
  return true;
}

struct SampleGrid {
  double x0, y0, cell;
  int nx, ny;
  const int* off;    // [nx*ny + 1]
  const int* idx;    // sample ids bucketed by cell
};

__global__ void k_lc_bounds(const double* s, int64_t ns, double* out) {
  // one block: min/max of the samples
  __shared__ double sh[4][256];
  double a = INFINITY, b = -INFINITY, c = INFINITY, d = -INFINITY;
  for (int64_t k = threadIdx.x; k < ns; k += blockDim.x) {
    a = fmin(a, s[2 * k]); b = fmax(b, s[2 * k]);
    c = fmin(c, s[2 * k + 1]); d = fmax(d, s[2 * k + 1]);
  }
  sh[0][threadIdx.x] = a; sh[1][threadIdx.x] = b; sh[2][threadIdx.x] = c; sh[3][threadIdx.x] = d;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] = fmin(sh[0][threadIdx.x], sh[0][threadIdx.x + o]);
      sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
      sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_lc_count(const double* s, int64_t ns, double x0, double y0, double cell, int nx,
                           int ny, int* cnt, int* cellof) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= ns) return;
  int cx = (int)floor((s[2 * k] - x0) / cell), cy = (int)floor((s[2 * k + 1] - y0) / cell);
  cx = min(max(cx, 0), nx - 1);
  cy = min(max(cy, 0), ny - 1);
  const int c = cy * nx + cx;
  cellof[k] = c;
  atomicAdd(&cnt[c], 1);
}

__global__ void k_lc_fill(int64_t ns, const int* cellof, const int* off, int* cur, int* idx) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const int c = cellof[k];
  idx[off[c] + atomicAdd(&cur[c], 1)] = (int)k;
}

// warp-aggregated atomicAdd of 1 (lanes with the same counter combine)
__device__ __forceinline__ unsigned long long agg_inc(unsigned long long* p, int key) {
  const unsigned grp = __match_any_sync(__activemask(), key);
  const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(p, (unsigned long long)__popc(grp));
  base = __shfl_sync(grp, base, leader);
  return base + __popc(grp & ((1u << lane) - 1u));
}

// rays within one cell of the sample grid: their cell in the grid widened by
// one cell on every side ((nx + 2) x (ny + 2)), -1 for the others
__global__ void k_lc_ray_cell(const double2* __restrict__ y, int64_t m, SampleGrid G,
                              int* __restrict__ cellof, unsigned long long* __restrict__ cnt) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const double2 p = y[r];
  const double fx = floor((p.x - G.x0) / G.cell), fy = floor((p.y - G.y0) / G.cell);
  if (fx >= -1.0 && fx <= (double)G.nx && fy >= -1.0 && fy <= (double)G.ny) {
    const int c = ((int)fy + 1) * (G.nx + 2) + (int)fx + 1;
    cellof[r] = c;
    agg_inc(&cnt[c], c);
  } else {
    cellof[r] = -1;
  }
}

__global__ void k_lc_ray_fill(const double2* __restrict__ y, int64_t m, const int* __restrict__ cellof,
                              const int64_t* __restrict__ off, unsigned long long* __restrict__ cur,
                              SampleGrid G, Pos* __restrict__ yp) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int c = cellof[r];
  if (c < 0) return;
  const int64_t pos = off[c] + (int64_t)agg_inc(&cur[c], c);
  const double2 p = y[r];
  const int nxe = G.nx + 2;
  const int cyw = c / nxe, cxw = c - cyw * nxe;  // widened cell: the grid's cell + 1
  yp[pos] = make_pos(p.x, p.y, cxw - 1, cyw - 1, G.x0, G.y0, G.cell);
}

// F_k: one block per sample over the bucketed rays of the 3 x 3 cells
__global__ void __launch_bounds__(kLcThreads)
k_lc_fwd(const double* __restrict__ s, int64_t ns, SampleGrid G, const int64_t* __restrict__ roff,
         const Pos* __restrict__ yp, ExpTab T, ff ninv2s2, ff cut2, float cutf, double norm,
         double* __restrict__ F) {
  __shared__ double red[kLcThreads / 32];
  const int64_t k = blockIdx.x;
  const double s1 = s[2 * k], s2 = s[2 * k + 1];
  int cx = (int)floor((s1 - G.x0) / G.cell), cy = (int)floor((s2 - G.y0) / G.cell);
  cx = min(max(cx, 0), G.nx - 1);
  cy = min(max(cy, 0), G.ny - 1);
  const Pos sp = make_pos(s1, s2, cx, cy, G.x0, G.y0, G.cell);
  const float side = (float)G.cell;
  const int nxe = G.nx + 2;
  ff acc{0.f, 0.f};
  for (int oy = 0; oy < 3; ++oy) {
    const int c0 = (cy + oy) * nxe + cx;  // cells (cx-1 .. cx+1, cy-1+oy) of the widened grid
    for (int64_t t = roff[c0] + threadIdx.x; t < roff[c0 + 3]; t += blockDim.x) {
      ff d1, d2, g;
      if (pair_gauss(yp[t], sp, side, cutf, ninv2s2, cut2, T, d1, d2, g)) acc = ff_add(acc, g);
    }
  }
  double a = ff_to_double(acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kLcThreads / 32; ++w) sum += red[w];
    F[k] = norm * sum;
  }
}

// samples in cell order: positions and the gradient coefficient
// 2 (F_k - T_k) norm (-1 / sigma^2) (float-float)
__global__ void k_lc_sample_coef(const double* __restrict__ s, const int* __restrict__ idx, int64_t ns,
                                 SampleGrid G, const double* __restrict__ F,
                                 const double* __restrict__ T, double coef0, Pos* __restrict__ sp,
                                 float2* __restrict__ coef) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ns) return;
  const int k = idx[t];
  const double s1 = s[2 * k], s2 = s[2 * k + 1];
  int cx = (int)floor((s1 - G.x0) / G.cell), cy = (int)floor((s2 - G.y0) / G.cell);
  cx = min(max(cx, 0), G.nx - 1);
  cy = min(max(cy, 0), G.ny - 1);
  sp[t] = make_pos(s1, s2, cx, cy, G.x0, G.y0, G.cell);
  const ff c = ff_of(2.0 * (F[k] - T[k]) * coef0);
  coef[t] = make_float2(c.hi, c.lo);
}

// dL/dy_r: one thread per ray over the samples of the 3 x 3 cells around it
__global__ void __launch_bounds__(kLcThreads)
k_lc_grad(const double* __restrict__ y, int64_t m, SampleGrid G, const Pos* __restrict__ sp,
          const float2* __restrict__ coef, ExpTab T, ff ninv2s2, ff cut2, float cutf,
          double* __restrict__ gy) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const double y1 = y[2 * r], y2 = y[2 * r + 1];
  const double fx = floor((y1 - G.x0) / G.cell), fy = floor((y2 - G.y0) / G.cell);
  ff g1{0.f, 0.f}, g2{0.f, 0.f};
  if (fx >= -1.0 && fx <= (double)G.nx && fy >= -1.0 && fy <= (double)G.ny) {
    const int cx = (int)fx, cy = (int)fy;
    const Pos yp = make_pos(y1, y2, cx, cy, G.x0, G.y0, G.cell);
    const float side = (float)G.cell;
    for (int oy = -1; oy <= 1; ++oy) {
      const int yy = cy + oy;
      if (yy < 0 || yy >= G.ny) continue;
      const int xa = max(cx - 1, 0), xb = min(cx + 1, G.nx - 1);
      if (xa > xb) continue;
      // cells xa .. xb of row yy are contiguous in the cell order
      for (int t = G.off[yy * G.nx + xa]; t < G.off[yy * G.nx + xb + 1]; ++t) {
        ff d1, d2, g;
        if (!pair_gauss(yp, sp[t], side, cutf, ninv2s2, cut2, T, d1, d2, g)) continue;
        const float2 c = coef[t];
        const ff c2 = ff_mul(ff{c.x, c.y}, g);
        g1 = ff_add(g1, ff_mul(c2, d1));
        g2 = ff_add(g2, ff_mul(c2, d2));
      }
    }
  }
  gy[2 * r] = ff_to_double(g1);
  gy[2 * r + 1] = ff_to_double(g2);
}

struct GridHolder {
  SampleGrid G;
  Scratch off, idx;
};

void build_sample_grid(const double* smp, int64_t ns, double sigma, double trunc, DeviceAlloc& da,
                       cudaStream_t s, GridHolder& H) {
  Scratch bb(&da, sizeof(double) * 4);
  k_lc_bounds<<<1, 256, 0, s>>>(smp, ns, bb.as<double>());
  LENS_LAUNCHED("k_lc_bounds");
  double hb[4];
  LENS_CUDA(cudaMemcpyAsync(hb, bb.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaStreamSynchronize(s));
  if (!(std::isfinite(hb[0]) && std::isfinite(hb[1]) && std::isfinite(hb[2]) && std::isfinite(hb[3])))
    fail(LENS_EINVAL, "non-finite light-curve sample");
  // side: the least k 2^e (k = 4 .. 8, three significant bits) at or above
  // trunc sigma; origin: a multiple of it.  Then a cell's origin x0 + i side
  // is exact in float64, and so is a point's offset from it.
  int ex = 0;
  std::frexp(trunc * sigma, &ex);  // trunc sigma in [2^(ex-1), 2^ex)
  const double unit = std::ldexp(1.0, ex - 3);
  double cell = std::ceil(trunc * sigma / unit) * unit;
  double x0 = 0, y0 = 0;
  int nx = 0, ny = 0;
  for (;;) {
    x0 = std::floor(hb[0] / cell) * cell;
    y0 = std::floor(hb[2] / cell) * cell;
    nx = (int)std::ceil((hb[1] - x0) / cell) + 1;
    ny = (int)std::ceil((hb[3] - y0) / cell) + 1;
    if ((int64_t)nx * ny <= (1 << 22)) break;
    cell *= 2.0;
  }
  const int nc = nx * ny;
  Scratch cnt(&da, sizeof(int64_t) * (nc + 1));
  Scratch off64(&da, sizeof(int64_t) * (nc + 1));
  Scratch cellof(&da, sizeof(int) * ns);
  H.off = Scratch(&da, sizeof(int) * (nc + 1));
  H.idx = Scratch(&da, sizeof(int) * ns);
  Scratch cnt32(&da, sizeof(int) * (nc + 1));
  LENS_CUDA(cudaMemsetAsync(cnt32.p, 0, cnt32.bytes, s));
  k_lc_count<<<grid_for(ns, 256), 256, 0, s>>>(smp, ns, x0, y0, cell, nx, ny,
                                               cnt32.as<int>(), cellof.as<int>());
  LENS_LAUNCHED("k_lc_count");
  // exclusive scan on the host side is fine for <= 4M cells? use device scan
  std::vector<int> hc(nc + 1);
  LENS_CUDA(cudaMemcpyAsync(hc.data(), cnt32.p, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaStreamSynchronize(s));
  std::vector<int> ho(nc + 1, 0);
  for (int c = 0; c < nc; ++c) ho[c + 1] = ho[c] + hc[c];
  LENS_CUDA(cudaMemcpyAsync(H.off.p, ho.data(), sizeof(int) * (nc + 1), cudaMemcpyHostToDevice, s));
  LENS_CUDA(cudaMemsetAsync(cnt32.p, 0, cnt32.bytes, s));
  k_lc_fill<<<grid_for(ns, 256), 256, 0, s>>>(ns, cellof.as<int>(), H.off.as<int>(),
                                              cnt32.as<int>(), H.idx.as<int>());
  LENS_LAUNCHED("k_lc_fill");
  LENS_CUDA(cudaStreamSynchronize(s));  // host vector ho must outlive the copy
  H.G = SampleGrid{x0, y0, cell, nx, ny, H.off.as<int>(), H.idx.as<int>()};
}

}  // namespace

void light_curve(const double* y, int64_t m, double w, const double* smp, int64_t ns,
                 double sigma, double trunc, double* F, cudaStream_t s) {
  DeviceAlloc da;
  da.stream = s;
  LENS_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * ns, s));
  if (m == 0 || ns == 0) return;
  GridHolder H;
  build_sample_grid(smp, ns, sigma, trunc, da, s, H);
  const SampleGrid& G = H.G;
  // the rays near the samples, bucketed over the widened sample grid
  const int64_t nce = (int64_t)(G.nx + 2) * (G.ny + 2);
  Scratch cellof(&da, sizeof(int) * (size_t)m);
  Scratch cnt(&da, sizeof(int64_t) * (size_t)(nce + 1)), off(&da, sizeof(int64_t) * (size_t)(nce + 1));
  Scratch cur(&da, sizeof(int64_t) * (size_t)(nce + 1));
  LENS_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes, s));
  LENS_CUDA(cudaMemsetAsync(cur.p, 0, cur.bytes, s));
  const double2* y2 = reinterpret_cast<const double2*>(y);
  k_lc_ray_cell<<<grid_for(m, 256), 256, 0, s>>>(y2, m, G, cellof.as<int>(),
                                                  cnt.as<unsigned long long>());
  LENS_LAUNCHED("k_lc_ray_cell");
  exclusive_scan_i64(cnt.as<int64_t>(), off.as<int64_t>(), nce + 1, da, s);
  int64_t near = 0;
  const int64_t* addr[1] = {off.as<int64_t>() + nce};
  read_i64(addr, 1, &near, da, s);
  Scratch yp(&da, sizeof(Pos) * (size_t)std::max<int64_t>(near, 1));
  k_lc_ray_fill<<<grid_for(m, 256), 256, 0, s>>>(y2, m, cellof.as<int>(), off.as<int64_t>(),
                                                  cur.as<unsigned long long>(), G, yp.as<Pos>());
  LENS_LAUNCHED("k_lc_ray_fill");
  if (ns > (int64_t)INT32_MAX) fail(LENS_EINVAL, "too many light-curve samples");
  static const ExpTab kExp = make_exp_tab();
  k_lc_fwd<<<(unsigned)ns, kLcThreads, 0, s>>>(smp, ns, G, off.as<int64_t>(), yp.as<Pos>(), kExp,
                                               ff_of(-1.0 / (2.0 * sigma * sigma)),
                                               ff_of(trunc * trunc * sigma * sigma),
                                               (float)(trunc * sigma),
                                               w / (2.0 * M_PI * sigma * sigma), F);
  LENS_LAUNCHED("k_lc_fwd");
  LENS_CUDA(cudaStreamSynchronize(s));
}

void light_curve_grad(const double* y, int64_t m, double w, const double* smp, int64_t ns,
                      double sigma, double trunc, const double* F, const double* T, double* gy,
                      cudaStream_t s) {
  DeviceAlloc da;
  da.stream = s;
  if (ns == 0) {
    LENS_CUDA(cudaMemsetAsync(gy, 0, sizeof(double) * 2 * m, s));
    return;
  }
  if (m == 0) return;
  GridHolder H;
  build_sample_grid(smp, ns, sigma, trunc, da, s, H);
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  const double norm = w / (2.0 * M_PI * sigma * sigma);
  Scratch sp(&da, sizeof(Pos) * (size_t)ns);
  Scratch coef(&da, sizeof(float2) * (size_t)ns);
  k_lc_sample_coef<<<grid_for(ns, 256), 256, 0, s>>>(smp, H.G.idx, ns, H.G, F, T,
                                                      norm * (-2.0 * inv2s2), sp.as<Pos>(),
                                                      coef.as<float2>());
  LENS_LAUNCHED("k_lc_sample_coef");
  static const ExpTab kExp = make_exp_tab();
  k_lc_grad<<<grid_for(m, kLcThreads), kLcThreads, 0, s>>>(y, m, H.G, sp.as<Pos>(),
                                                           coef.as<float2>(), kExp, ff_of(-inv2s2),
                                                           ff_of(trunc * trunc * sigma * sigma),
                                                           (float)(trunc * sigma), gy);
  LENS_LAUNCHED("k_lc_grad");
  LENS_CUDA(cudaStreamSynchronize(s));
}

}  // namespace lens
