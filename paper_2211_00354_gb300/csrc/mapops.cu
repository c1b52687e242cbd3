// mapops.cu -- consumers of a magnification map (Sec. 3: magnification
// histograms of finite sources, light curves along source tracks).
//  * finite Gaussian source: the map convolved with a Gaussian truncated at R
//    pixels along each axis and renormalised to the part of the kernel inside
//    the map; the window is a rectangle, so numerator and normalisation are
//    both separable: one pass along rows, one along columns, thread per
//    output pixel, float64;
//  * histogram: equal bins of the value or of log10(value), counts kept per
//    block in shared memory, then one atomic per bin and block;
//  * track: the map bilinear between pixel centres at source positions.
#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kMaxSourceRadius = 1024;  // pixels

// pass along x: t[p] = sum_{|dx| <= R, in map} w[|dx|] map[p + dx]
__global__ void k_source_rows(const double* __restrict__ map, int npx, int npy, int R,
                              const double* __restrict__ w, double* __restrict__ t) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)npx * npy) return;
  const int py = (int)(i / npx), px = (int)(i - (int64_t)py * npx);
  const double* row = map + (int64_t)py * npx;
  const int a = max(px - R, 0), b = min(px + R, npx - 1);
  double s = 0.0;
  for (int q = a; q <= b; ++q) s = fma(w[abs(q - px)], row[q], s);
  t[i] = s;
}

// pass along y, divided by the in-map kernel weight (a product of the two
// axes' in-map sums)
__global__ void k_source_cols(const double* __restrict__ t, int npx, int npy, int R,
                              const double* __restrict__ w, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)npx * npy) return;
  const int py = (int)(i / npx), px = (int)(i - (int64_t)py * npx);
  const int a = max(py - R, 0), b = min(py + R, npy - 1);
  double s = 0.0, wy = 0.0;
  for (int q = a; q <= b; ++q) {
    const double wq = w[abs(q - py)];
    s = fma(wq, t[(int64_t)q * npx + px], s);
    wy += wq;
  }
  const int ax = max(px - R, 0), bx = min(px + R, npx - 1);
  double wx = 0.0;
  for (int q = ax; q <= bx; ++q) wx += w[abs(q - px)];
  out[i] = s / (wx * wy);
}

__global__ void k_histogram(const double* __restrict__ v, int64_t n, double lo, double hi,
                            int nbins, int log_bins, unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned int hb[];  // nbins + 2
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x) hb[b] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x = v[i];
    int b;
    if (log_bins && !(x > 0.0)) {
      b = 0;
    } else {
      if (log_bins) x = log10(x);
      if (x < lo) b = 0;
      else if (x >= hi) b = nbins + 1;
      else b = 1 + min((int)floor((x - lo) / (hi - lo) * nbins), nbins - 1);
    }
    atomicAdd(&hb[b], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x)
    if (hb[b]) atomicAdd(&counts[b], (unsigned long long)hb[b]);
}

__global__ void k_track(const double* __restrict__ map, int npx, int npy, double u0, double v0,
                        double du, double dv, const double2* __restrict__ s, int64_t ns,
                        double* __restrict__ out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= ns) return;
  double x = (s[k].x - u0) / du - 0.5, y = (s[k].y - v0) / dv - 0.5;
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

}  // namespace

void map_source(const double* map, int npx, int npy, double sigma_px, double trunc, double* out,
                DeviceAlloc& da, cudaStream_t s) {
  const int R = (int)std::floor(trunc * sigma_px);
  if (R > kMaxSourceRadius) fail(LENS_EINVAL, "source radius above 1024 pixels");
  std::vector<double> w((size_t)R + 1);
  const double inv2s2 = 1.0 / (2.0 * sigma_px * sigma_px);
  for (int d = 0; d <= R; ++d) w[(size_t)d] = std::exp(-(double)d * d * inv2s2);
  Scratch dw(&da, sizeof(double) * w.size());
  Scratch t(&da, sizeof(double) * (size_t)npx * (size_t)npy);
  LENS_CUDA(cudaMemcpyAsync(dw.p, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, s));
  const int64_t n = (int64_t)npx * npy;
  k_source_rows<<<grid_for(n, 256), 256, 0, s>>>(map, npx, npy, R, dw.as<double>(), t.as<double>());
  LENS_LAUNCHED("k_source_rows");
  k_source_cols<<<grid_for(n, 256), 256, 0, s>>>(t.as<double>(), npx, npy, R, dw.as<double>(), out);
  LENS_LAUNCHED("k_source_cols");
  // the host weights must outlive the copy
  LENS_CUDA(cudaStreamSynchronize(s));
}

void map_histogram(const double* v, int64_t n, double lo, double hi, int nbins, int log_bins,
                   int64_t* counts, cudaStream_t s) {
  LENS_CUDA(cudaMemsetAsync(counts, 0, sizeof(int64_t) * (size_t)(nbins + 2), s));
  if (n == 0) return;
  const size_t smem = sizeof(unsigned int) * (size_t)(nbins + 2);
  k_histogram<<<grid_for(n, 256, 152 * 8), 256, smem, s>>>(
      v, n, lo, hi, nbins, log_bins, reinterpret_cast<unsigned long long*>(counts));
  LENS_LAUNCHED("k_histogram");
}

void map_track(const double* map, int npx, int npy, const double box[4], const double* pos,
               int64_t ns, double* out, cudaStream_t s) {
  if (ns == 0) return;
  const double du = (box[1] - box[0]) / npx, dv = (box[3] - box[2]) / npy;
  k_track<<<grid_for(ns, 256), 256, 0, s>>>(map, npx, npy, box[0], box[2], du, dv,
                                            reinterpret_cast<const double2*>(pos), ns, out);
  LENS_LAUNCHED("k_track");
}

}  // namespace lens
