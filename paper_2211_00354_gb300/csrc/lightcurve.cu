// lightcurve.cu -- Gaussian-source light curve as a ray sum and its gradient
// with respect to the mapped rays.  A source of profile
// G(s) = exp(-|s|^2 / (2 sigma^2)) / (2 pi sigma^2) (the Gaussian source of
// Sec. 2.5) centred at s_k has magnification F_k = sum_r w_ray G(y_r - s_k)
// when every ray carries the image-plane area w_ray; sampling s_k along a
// track gives a light curve (Sec. 3.3).  Pairs with |y_r - s_k| > trunc sigma
// are left out.  L = sum_k (F_k - T_k)^2 gives
//   dL/dy_r = sum_k 2 (F_k - T_k) w_ray G(y_r - s_k) (-(y_r - s_k) / sigma^2).
// Samples are bucketed on a uniform grid of cell trunc*sigma, so each ray
// visits only the 3 x 3 cells around it.  Float64 throughout.
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

template <bool GRAD>
__global__ void __launch_bounds__(kLcThreads)
k_lc(const double* __restrict__ y, int64_t m, double w, const double* __restrict__ s, int64_t ns,
     double sigma, double trunc, SampleGrid G, double* __restrict__ F,
     const double* __restrict__ Fin, const double* __restrict__ T, double* __restrict__ gy) {
  extern __shared__ double sF[];  // forward: per-block partial light curve
  if (!GRAD) {
    for (int64_t k = threadIdx.x; k < ns; k += blockDim.x) sF[k] = 0.0;
    __syncthreads();
  }
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  const double norm = w / (2.0 * M_PI * sigma * sigma);
  const double cut2 = trunc * trunc * sigma * sigma;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double y1 = y[2 * r], y2 = y[2 * r + 1];
    const double fx = floor((y1 - G.x0) / G.cell), fy = floor((y2 - G.y0) / G.cell);
    double g1 = 0.0, g2 = 0.0;
    if (fx >= -1.0 && fx <= (double)G.nx && fy >= -1.0 && fy <= (double)G.ny) {
      const int cx = (int)fx, cy = (int)fy;
      for (int oy = -1; oy <= 1; ++oy) {
        const int yy = cy + oy;
        if (yy < 0 || yy >= G.ny) continue;
        for (int ox = -1; ox <= 1; ++ox) {
          const int xx = cx + ox;
          if (xx < 0 || xx >= G.nx) continue;
          const int c = yy * G.nx + xx;
          for (int t = G.off[c]; t < G.off[c + 1]; ++t) {
            const int k = G.idx[t];
            const double d1 = y1 - s[2 * k], d2 = y2 - s[2 * k + 1];
            const double q = d1 * d1 + d2 * d2;
            if (q > cut2) continue;
            const double e = exp(-q * inv2s2);
            if (!GRAD) {
              atomicAdd(&sF[k], e);
            } else {
              const double c2 = 2.0 * (Fin[k] - T[k]) * norm * e * (-2.0 * inv2s2);
              g1 += c2 * d1;
              g2 += c2 * d2;
            }
          }
        }
      }
    }
    if (GRAD) { gy[2 * r] = g1; gy[2 * r + 1] = g2; }
  }
  if (!GRAD) {
    __syncthreads();
    for (int64_t k = threadIdx.x; k < ns; k += blockDim.x)
      if (sF[k] != 0.0) atomicAdd(&F[k], norm * sF[k]);
  }
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
  if (m == 0) return;
  if (ns > 6000) fail(LENS_EINVAL, "at most 6000 light-curve samples per call");
  GridHolder H;
  build_sample_grid(smp, ns, sigma, trunc, da, s, H);
  const size_t smem = sizeof(double) * ns;
  if (smem > 48 * 1024)
    LENS_CUDA(cudaFuncSetAttribute(k_lc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_lc<false><<<grid_for(m, kLcThreads, 152 * 8), kLcThreads, smem, s>>>(
      y, m, w, smp, ns, sigma, trunc, H.G, F, nullptr, nullptr, nullptr);
  LENS_LAUNCHED("k_lc<forward>");
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
  GridHolder H;
  build_sample_grid(smp, ns, sigma, trunc, da, s, H);
  k_lc<true><<<grid_for(m, kLcThreads), kLcThreads, 0, s>>>(y, m, w, smp, ns, sigma, trunc, H.G,
                                                            nullptr, F, T, gy);
  LENS_LAUNCHED("k_lc<grad>");
  LENS_CUDA(cudaStreamSynchronize(s));
}

}  // namespace lens
