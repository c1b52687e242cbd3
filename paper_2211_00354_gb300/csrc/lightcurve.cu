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
// with their coefficients.  A pair's cut test and Gaussian are float64; a
// float32 test with a margin for its rounding skips the float64 work for
// pairs clearly beyond the cut (GB300's float64 pipe is 1/74 of float32).
#include <algorithm>
#include <cmath>
#include <vector>

#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kLcThreads = 256;

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

// Could the pair (y, s) be within the cut?  float32 copies of y and s carry
// an absolute error of at most 2^-24 (|y| + |s|) per coordinate, which the
// threshold absorbs (together with the rounding of d and q); false only for
// pairs surely beyond the cut.
__device__ __forceinline__ bool maybe_within(float2 yf, float2 sf, float cut) {
  const float d1 = yf.x - sf.x, d2 = yf.y - sf.y;
  const float e = 2.4e-7f * (fabsf(yf.x) + fabsf(yf.y) + fabsf(sf.x) + fabsf(sf.y)) + 1e-30f;
  const float c = cut * 1.00001f + 4.f * e;
  return fmaf(d1, d1, d2 * d2) <= c * c;
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
                              double2* __restrict__ yd, float2* __restrict__ yf) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int c = cellof[r];
  if (c < 0) return;
  const int64_t pos = off[c] + (int64_t)agg_inc(&cur[c], c);
  const double2 p = y[r];
  yd[pos] = p;
  yf[pos] = make_float2((float)p.x, (float)p.y);
}

// F_k: one block per sample over the bucketed rays of the 3 x 3 cells
__global__ void __launch_bounds__(kLcThreads)
k_lc_fwd(const double* __restrict__ s, int64_t ns, SampleGrid G, const int64_t* __restrict__ roff,
         const double2* __restrict__ yd, const float2* __restrict__ yf, double inv2s2,
         double cut2, float cutf, double norm, double* __restrict__ F) {
  __shared__ double red[kLcThreads / 32];
  const int64_t k = blockIdx.x;
  const double s1 = s[2 * k], s2 = s[2 * k + 1];
  const float2 sf = make_float2((float)s1, (float)s2);
  int cx = (int)floor((s1 - G.x0) / G.cell), cy = (int)floor((s2 - G.y0) / G.cell);
  cx = min(max(cx, 0), G.nx - 1);
  cy = min(max(cy, 0), G.ny - 1);
  const int nxe = G.nx + 2;
  double acc = 0.0;
  for (int oy = 0; oy < 3; ++oy) {
    const int c0 = (cy + oy) * nxe + cx;  // cells (cx-1 .. cx+1, cy-1+oy) of the widened grid
    for (int64_t t = roff[c0] + threadIdx.x; t < roff[c0 + 3]; t += blockDim.x) {
      if (!maybe_within(yf[t], sf, cutf)) continue;
      const double2 p = yd[t];
      const double d1 = p.x - s1, d2 = p.y - s2;
      const double q = d1 * d1 + d2 * d2;
      if (q > cut2) continue;
      acc += exp(-q * inv2s2);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kLcThreads / 32; ++w) sum += red[w];
    F[k] = norm * sum;
  }
}

// samples in cell order: positions (float64 and float32) and the gradient
// coefficient 2 (F_k - T_k) norm (-1 / sigma^2)
__global__ void k_lc_sample_coef(const double* __restrict__ s, const int* __restrict__ idx, int64_t ns,
                                 const double* __restrict__ F, const double* __restrict__ T,
                                 double coef0, double2* __restrict__ sd, float2* __restrict__ sfo,
                                 double* __restrict__ coef) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ns) return;
  const int k = idx[t];
  const double2 p = make_double2(s[2 * k], s[2 * k + 1]);
  sd[t] = p;
  sfo[t] = make_float2((float)p.x, (float)p.y);
  coef[t] = 2.0 * (F[k] - T[k]) * coef0;
}

// dL/dy_r: one thread per ray over the samples of the 3 x 3 cells around it
__global__ void __launch_bounds__(kLcThreads)
k_lc_grad(const double* __restrict__ y, int64_t m, SampleGrid G, const double2* __restrict__ sd,
          const float2* __restrict__ sfo, const double* __restrict__ coef, double inv2s2,
          double cut2, float cutf, double* __restrict__ gy) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const double y1 = y[2 * r], y2 = y[2 * r + 1];
  const float2 yf = make_float2((float)y1, (float)y2);
  const double fx = floor((y1 - G.x0) / G.cell), fy = floor((y2 - G.y0) / G.cell);
  double g1 = 0.0, g2 = 0.0;
  if (fx >= -1.0 && fx <= (double)G.nx && fy >= -1.0 && fy <= (double)G.ny) {
    const int cx = (int)fx, cy = (int)fy;
    for (int oy = -1; oy <= 1; ++oy) {
      const int yy = cy + oy;
      if (yy < 0 || yy >= G.ny) continue;
      const int xa = max(cx - 1, 0), xb = min(cx + 1, G.nx - 1);
      if (xa > xb) continue;
      // cells xa .. xb of row yy are contiguous in the cell order
      for (int t = G.off[yy * G.nx + xa]; t < G.off[yy * G.nx + xb + 1]; ++t) {
        if (!maybe_within(yf, sfo[t], cutf)) continue;
        const double2 p = sd[t];
        const double d1 = y1 - p.x, d2 = y2 - p.y;
        const double q = d1 * d1 + d2 * d2;
        if (q > cut2) continue;
        const double c2 = coef[t] * exp(-q * inv2s2);
        g1 += c2 * d1;
        g2 += c2 * d2;
      }
    }
  }
  gy[2 * r] = g1;
  gy[2 * r + 1] = g2;
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
  double cell = trunc * sigma;
  int nx = (int)std::ceil((hb[1] - hb[0]) / cell) + 1, ny = (int)std::ceil((hb[3] - hb[2]) / cell) + 1;
  while ((int64_t)nx * ny > (1 << 22)) {
    cell *= 2.0;
    nx = (int)std::ceil((hb[1] - hb[0]) / cell) + 1;
    ny = (int)std::ceil((hb[3] - hb[2]) / cell) + 1;
  }
  const int nc = nx * ny;
  Scratch cnt(&da, sizeof(int64_t) * (nc + 1));
  Scratch off64(&da, sizeof(int64_t) * (nc + 1));
  Scratch cellof(&da, sizeof(int) * ns);
  H.off = Scratch(&da, sizeof(int) * (nc + 1));
  H.idx = Scratch(&da, sizeof(int) * ns);
  Scratch cnt32(&da, sizeof(int) * (nc + 1));
  LENS_CUDA(cudaMemsetAsync(cnt32.p, 0, cnt32.bytes, s));
  k_lc_count<<<grid_for(ns, 256), 256, 0, s>>>(smp, ns, hb[0], hb[2], cell, nx, ny,
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
  H.G = SampleGrid{hb[0], hb[2], cell, nx, ny, H.off.as<int>(), H.idx.as<int>()};
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
  Scratch yd(&da, sizeof(double2) * (size_t)std::max<int64_t>(near, 1));
  Scratch yf(&da, sizeof(float2) * (size_t)std::max<int64_t>(near, 1));
  k_lc_ray_fill<<<grid_for(m, 256), 256, 0, s>>>(y2, m, cellof.as<int>(), off.as<int64_t>(),
                                                  cur.as<unsigned long long>(), yd.as<double2>(),
                                                  yf.as<float2>());
  LENS_LAUNCHED("k_lc_ray_fill");
  if (ns > (int64_t)INT32_MAX) fail(LENS_EINVAL, "too many light-curve samples");
  k_lc_fwd<<<(unsigned)ns, kLcThreads, 0, s>>>(smp, ns, G, off.as<int64_t>(), yd.as<double2>(),
                                               yf.as<float2>(), 1.0 / (2.0 * sigma * sigma),
                                               trunc * trunc * sigma * sigma,
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
  Scratch sd(&da, sizeof(double2) * (size_t)ns), sf(&da, sizeof(float2) * (size_t)ns);
  Scratch coef(&da, sizeof(double) * (size_t)ns);
  k_lc_sample_coef<<<grid_for(ns, 256), 256, 0, s>>>(smp, H.G.idx, ns, F, T, norm * (-2.0 * inv2s2),
                                                      sd.as<double2>(), sf.as<float2>(),
                                                      coef.as<double>());
  LENS_LAUNCHED("k_lc_sample_coef");
  k_lc_grad<<<grid_for(m, kLcThreads), kLcThreads, 0, s>>>(y, m, H.G, sd.as<double2>(),
                                                           sf.as<float2>(), coef.as<double>(),
                                                           inv2s2, trunc * trunc * sigma * sigma,
                                                           (float)(trunc * sigma), gy);
  LENS_LAUNCHED("k_lc_grad");
  LENS_CUDA(cudaStreamSynchronize(s));
}

}  // namespace lens
