// direct.cu -- Eq. 1 by O(N* x N_x) direct summation (Sec. 2.1): the GPU
// baseline the FMM is measured against.
//
// FP32 form: every position is split once into a float pair (hi, lo) with
// hi + lo == x to ~48 bits, and a pair difference is taken as
// (hi_r - hi_s) + (lo_r - lo_s).  When a star is close to a ray the hi
// difference is exact (Sterbenz), so the near terms keep float32 relative
// accuracy even at |x| ~ 1e3 Einstein radii.  Each shared-memory tile of stars
// is summed in plain float32 and the tile partial is added to a two-sum
// (hi, lo) accumulator.  y = diag(a, b) x - alpha is formed in float64.
// FP64 form: the same loop in float64 with per-tile partials.
#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kThreads = 128;
constexpr int kTile = 256;

__global__ void k_split_stars(const double* __restrict__ stars, const double* __restrict__ m,
                              int64_t n, float4* __restrict__ hl, float* __restrict__ mf) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = stars[2 * i], y = stars[2 * i + 1];
  float xh = (float)x, yh = (float)y;
  hl[i] = make_float4(xh, yh, (float)(x - (double)xh), (float)(y - (double)yh));
  mf[i] = (float)m[i];
}

template <int RPT, bool JAC>
__global__ void __launch_bounds__(kThreads)
k_direct_f32(const float4* __restrict__ shl, const float* __restrict__ sm, int64_t n,
             const double* __restrict__ rays, int64_t m, double a, double b,
             double* __restrict__ y, double* __restrict__ jac) {
  __shared__ float4 t_pos[kTile];
  __shared__ float t_m[kTile];
  const int64_t base = (int64_t)blockIdx.x * kThreads * RPT;
  float rxh[RPT], ryh[RPT], rxl[RPT], ryl[RPT];
  fcomp ax[RPT], ay[RPT];
  fcomp j11[RPT], j12[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    int64_t r = base + threadIdx.x + (int64_t)k * kThreads;
    double x1 = 0, x2 = 0;
    if (r < m) { x1 = rays[2 * r]; x2 = rays[2 * r + 1]; }
    rxh[k] = (float)x1; ryh[k] = (float)x2;
    rxl[k] = (float)(x1 - (double)rxh[k]); ryl[k] = (float)(x2 - (double)ryh[k]);
    ax[k] = {0.f, 0.f}; ay[k] = {0.f, 0.f}; j11[k] = {0.f, 0.f}; j12[k] = {0.f, 0.f};
  }
  for (int64_t t0 = 0; t0 < n; t0 += kTile) {
    const int cnt = (int)min64(kTile, n - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += kThreads) { t_pos[q] = shl[t0 + q]; t_m[q] = sm[t0 + q]; }
    __syncthreads();
    float px[RPT], py[RPT], pj11[RPT], pj12[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) { px[k] = 0.f; py[k] = 0.f; pj11[k] = 0.f; pj12[k] = 0.f; }
    for (int q = 0; q < cnt; ++q) {
      const float4 s = t_pos[q];
      const float ms = t_m[q];
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const float d1 = (rxh[k] - s.x) + (rxl[k] - s.z);
        const float d2 = (ryh[k] - s.y) + (ryl[k] - s.w);
        // a star exactly on the ray contributes nothing: without the
        // Jacobian a tiny floor on r2 does it (w * d = 0 with w finite),
        // with it the select (w * w would overflow)
        const float r2 = JAC ? fmaf(d1, d1, d2 * d2) : fmaf(d1, d1, fmaf(d2, d2, 1e-30f));
        const float inv = JAC ? (r2 > 0.f ? frcp_fast(r2) : 0.f) : frcp_fast(r2);
        const float w = ms * inv;
        px[k] = fmaf(w, d1, px[k]);
        py[k] = fmaf(w, d2, py[k]);
        if (JAC) {
          const float w2 = w * inv;
          pj11[k] = fmaf(w2, (d2 - d1) * (d2 + d1), pj11[k]);
          pj12[k] = fmaf(w2, -2.f * d1 * d2, pj12[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      ax[k].add(px[k]); ay[k].add(py[k]);
      if (JAC) { j11[k].add(pj11[k]); j12[k].add(pj12[k]); }
    }
  }
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    int64_t r = base + threadIdx.x + (int64_t)k * kThreads;
    if (r >= m) continue;
    const double x1 = rays[2 * r], x2 = rays[2 * r + 1];
    y[2 * r] = fma(a, x1, -ax[k].value());
    y[2 * r + 1] = fma(b, x2, -ay[k].value());
    if (JAC) {
      const double d11 = j11[k].value(), d12 = j12[k].value();
      jac[4 * r + 0] = a - d11;
      jac[4 * r + 1] = -d12;
      jac[4 * r + 2] = -d12;
      jac[4 * r + 3] = b + d11;
    }
  }
}

template <bool JAC>
__global__ void __launch_bounds__(kThreads)
k_direct_f64(const double* __restrict__ stars, const double* __restrict__ sm, int64_t n,
             const double* __restrict__ rays, int64_t m, double a, double b,
             double* __restrict__ y, double* __restrict__ jac) {
  __shared__ double2 t_pos[kTile];
  __shared__ double t_m[kTile];
  const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  double x1 = 0, x2 = 0;
  if (r < m) { x1 = rays[2 * r]; x2 = rays[2 * r + 1]; }
  double ax = 0, ay = 0, cx = 0, cy = 0, s11 = 0, s12 = 0;
  for (int64_t t0 = 0; t0 < n; t0 += kTile) {
    const int cnt = (int)min64(kTile, n - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += kThreads) {
      t_pos[q] = make_double2(stars[2 * (t0 + q)], stars[2 * (t0 + q) + 1]);
      t_m[q] = sm[t0 + q];
    }
    __syncthreads();
    double px = 0, py = 0;
    for (int q = 0; q < cnt; ++q) {
      const double d1 = x1 - t_pos[q].x, d2 = x2 - t_pos[q].y;
      const double r2 = d1 * d1 + d2 * d2;
      if (r2 == 0.0) continue;
      const double inv = 1.0 / r2;
      const double w = t_m[q] * inv;
      px = fma(w, d1, px);
      py = fma(w, d2, py);
      if (JAC) {
        const double w2 = w * inv;
        s11 = fma(w2, (d2 - d1) * (d2 + d1), s11);
        s12 = fma(w2, -2.0 * d1 * d2, s12);
      }
    }
    // Neumaier step for the tile partials
    double t = ax + px;
    cx += fabs(ax) >= fabs(px) ? (ax - t) + px : (px - t) + ax;
    ax = t;
    t = ay + py;
    cy += fabs(ay) >= fabs(py) ? (ay - t) + py : (py - t) + ay;
    ay = t;
  }
  if (r >= m) return;
  y[2 * r] = fma(a, x1, -(ax + cx));
  y[2 * r + 1] = fma(b, x2, -(ay + cy));
  if (JAC) {
    jac[4 * r + 0] = a - s11;
    jac[4 * r + 1] = -s12;
    jac[4 * r + 2] = -s12;
    jac[4 * r + 3] = b + s11;
  }
}

}  // namespace

void direct_deflect(const double* stars, const double* masses, int64_t n, double ks,
                    double g, const double* rays, int64_t m, int prec, double* y,
                    double* jac, DeviceAlloc& da, cudaStream_t s) {
  const double a = 1.0 - ks - g, b = 1.0 - ks + g;
  if (m == 0) return;
  if (prec == LENS_FP64) {
    if (jac) k_direct_f64<true><<<grid_for(m, kThreads), kThreads, 0, s>>>(stars, masses, n, rays, m, a, b, y, jac);
    else k_direct_f64<false><<<grid_for(m, kThreads), kThreads, 0, s>>>(stars, masses, n, rays, m, a, b, y, jac);
    LENS_LAUNCHED("k_direct_f64");
    return;
  }
  Scratch hl(&da, sizeof(float4) * (size_t)n), mf(&da, sizeof(float) * (size_t)n);
  k_split_stars<<<grid_for(n, 256), 256, 0, s>>>(stars, masses, n, hl.as<float4>(), mf.as<float>());
  LENS_LAUNCHED("k_split_stars");
  constexpr int RPT = 4;
  const unsigned blocks = grid_for(m, kThreads * RPT);
  if (jac) k_direct_f32<RPT, true><<<blocks, kThreads, 0, s>>>(hl.as<float4>(), mf.as<float>(), n, rays, m, a, b, y, jac);
  else k_direct_f32<RPT, false><<<blocks, kThreads, 0, s>>>(hl.as<float4>(), mf.as<float>(), n, rays, m, a, b, y, jac);
  LENS_LAUNCHED("k_direct_f32");
}

// The float32 direct sum with caller-provided scratch for the split stars
// (n float4 + n float); used by the allocation-free entry point.
void direct_f32_into(const double* stars, const double* masses, int64_t n, double ks, double g,
                     const double* rays, int64_t m, double* y, double* jac, float4* hl, float* mf,
                     cudaStream_t s) {
  const double a = 1.0 - ks - g, b = 1.0 - ks + g;
  if (m == 0) return;
  k_split_stars<<<grid_for(n, 256), 256, 0, s>>>(stars, masses, n, hl, mf);
  LENS_LAUNCHED("k_split_stars");
  constexpr int RPT = 4;
  const unsigned blocks = grid_for(m, kThreads * RPT);
  if (jac) k_direct_f32<RPT, true><<<blocks, kThreads, 0, s>>>(hl, mf, n, rays, m, a, b, y, jac);
  else k_direct_f32<RPT, false><<<blocks, kThreads, 0, s>>>(hl, mf, n, rays, m, a, b, y, jac);
  LENS_LAUNCHED("k_direct_f32");
}

}  // namespace lens
