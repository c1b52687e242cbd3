// mapops.cu -- consumers of a magnification map (Sec. 3: magnification
// histograms of finite sources, light curves along source tracks).
//  * finite Gaussian source: the map seen by a circular Gaussian source of
//    sigma pixels whose profile is cut at the isophote |d| = trunc sigma,
//    renormalised to the part of the profile inside the map.  The disk is a
//    stack of row segments |dx| <= r(dy); the weight exp(-|d|^2 / 2 s^2) is
//    g(dx) g(dy), so each output pixel sums, per dy >= 0, the two map rows
//    y + dy and y - dy (added once into shared memory) against g(dx) over
//    |dx| <= r(dy), folded as g(0) T[x] + sum_k g(k) (T[x+k] + T[x-k]); the
//    normalisation is the same stack of segments over the all-ones map, a
//    prefix sum of g per segment (one constant for the pixels at least R from
//    every edge).  Block per 256 pixels of a row; the map and g are taken
//    as float-float (pairs of float32, ~48 bits) and the sums run on the
//    float32 pipe (GB300's float64 pipe is ~1/64 of it), the normalisation
//    and the quotient in float64;
//  * histogram: equal bins of the value or of log10(value), counts kept per
//    block in shared memory, then one atomic per bin and block;
//  * track: the map bilinear between pixel centres at source positions.
#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kMaxSourceRadius = 1024;  // pixels
constexpr int kSourceThreads = 256;

// the map as float-float
__global__ void k_map_ff(const double* __restrict__ map, int64_t n, float2* __restrict__ mf) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ff v = ff_of(map[i]);
  mf[i] = make_float2(v.hi, v.lo);
}

// tab: g[0..R] (g[k] = exp(-k^2 / 2 s^2)), G[0..R] (G[k] = g[0] + .. + g[k]),
// then r[0..R] as ints (r[dy]: largest |dx| with dx^2 + dy^2 <= (trunc s)^2,
// -1 if none).  dfull: the normalisation of a pixel at least R from every
// edge.  Shared memory: g as float-float, then the folded row T (256 + 2 R).
__global__ void __launch_bounds__(kSourceThreads)
k_source_disk(const float2* __restrict__ mf, int npx, int npy, int R,
              const double* __restrict__ tab, double dfull, double* __restrict__ out) {
  extern __shared__ float2 smf[];
  float2* gf = smf;
  float2* T = smf + (R + 1);
  const double* G = tab + (R + 1);
  const int* rt = reinterpret_cast<const int*>(tab + 2 * (R + 1));
  const int t = threadIdx.x;
  const int blocks_x = (npx + kSourceThreads - 1) / kSourceThreads;
  const int py = blockIdx.x / blocks_x;
  const int x0 = (blockIdx.x - py * blocks_x) * kSourceThreads;
  const int px = x0 + t;
  for (int k = t; k <= R; k += kSourceThreads) {
    const ff v = ff_of(tab[k]);
    gf[k] = make_float2(v.hi, v.lo);
  }
  // every pixel of the block at least R from every edge: one normalisation
  const bool interior = x0 >= R && x0 + kSourceThreads - 1 <= npx - 1 - R && py >= R &&
                        py <= npy - 1 - R;
  ff num{0.f, 0.f};
  double den = 0.0;
  for (int dy = 0; dy <= R; ++dy) {
    const int r = rt[dy];
    const int ya = py + dy, yb = py - dy;
    const bool ina = ya < npy, inb = dy > 0 && yb >= 0;
    if (r < 0 || !(ina || inb)) continue;  // uniform over the block
    __syncthreads();  // the previous segment's readers of T are done
    const int nt = kSourceThreads + 2 * r;
    for (int i = t; i < nt; i += kSourceThreads) {
      const int x = x0 - r + i;
      ff v{0.f, 0.f};
      if (x >= 0 && x < npx) {
        if (ina) { const float2 a = mf[(int64_t)ya * npx + x]; v = ff{a.x, a.y}; }
        if (inb) { const float2 b = mf[(int64_t)yb * npx + x]; v = ff_add(v, ff{b.x, b.y}); }
      }
      T[i] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    if (px < npx) {
      const int c = t + r;
      ff acc = ff_mul(ff{gf[0].x, gf[0].y}, ff{T[c].x, T[c].y});
      for (int k = 1; k <= r; ++k) {
        const ff pair = ff_add(ff{T[c + k].x, T[c + k].y}, ff{T[c - k].x, T[c - k].y});
        acc = ff_add(acc, ff_mul(ff{gf[k].x, gf[k].y}, pair));
      }
      num = ff_add(num, ff_mul(ff{gf[dy].x, gf[dy].y}, acc));
      if (!interior) {
        // in-map weight of this segment: columns px - min(r, px) .. px + min(r, npx-1-px)
        const double seg = G[min(r, px)] + G[min(r, npx - 1 - px)] - tab[0];
        den = fma(tab[dy] * ((ina ? 1.0 : 0.0) + (inb ? 1.0 : 0.0)), seg, den);
      }
    }
  }
  if (px < npx) out[(int64_t)py * npx + px] = ff_to_double(num) / (interior ? dfull : den);
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
  // the disk: integer offsets with dx^2 + dy^2 <= (trunc sigma)^2 (the same
  // products in the same order as the definition, so the same offsets)
  const double cut2 = trunc * trunc * sigma_px * sigma_px;
  const double inv2s2 = 1.0 / (2.0 * sigma_px * sigma_px);
  const size_t n1 = (size_t)R + 1;
  std::vector<double> tab(3 * n1, 0.0);
  double acc = 0.0;
  for (int d = 0; d <= R; ++d) {
    tab[(size_t)d] = std::exp(-(double)d * d * inv2s2);
    acc += tab[(size_t)d];
    tab[n1 + (size_t)d] = acc;
  }
  int* rt = reinterpret_cast<int*>(tab.data() + 2 * n1);
  for (int dy = 0; dy <= R; ++dy) {
    int r = -1;
    while (r < R && (double)(r + 1) * (r + 1) + (double)dy * dy <= cut2) ++r;
    rt[dy] = r;
  }
  // the normalisation of an interior pixel, in the kernel's order
  double dfull = 0.0;
  for (int dy = 0; dy <= R; ++dy) {
    if (rt[dy] < 0) continue;
    const double seg = tab[n1 + (size_t)rt[dy]] + tab[n1 + (size_t)rt[dy]] - tab[0];
    dfull = std::fma(tab[(size_t)dy] * (dy > 0 ? 2.0 : 1.0), seg, dfull);
  }
  Scratch dt(&da, sizeof(double) * tab.size());
  LENS_CUDA(cudaMemcpyAsync(dt.p, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice,
                            s));
  const int64_t npix = (int64_t)npx * npy;
  Scratch mf(&da, sizeof(float2) * (size_t)npix);
  k_map_ff<<<grid_for(npix, 256), 256, 0, s>>>(map, npix, mf.as<float2>());
  LENS_LAUNCHED("k_map_ff");
  const int blocks_x = (npx + kSourceThreads - 1) / kSourceThreads;
  const int64_t blocks = (int64_t)blocks_x * npy;
  if (blocks > INT32_MAX) fail(LENS_EINVAL, "map too large");
  const size_t smem = sizeof(float2) * (n1 + kSourceThreads + 2 * (size_t)R);
  if (smem > 48 * 1024)
    LENS_CUDA(cudaFuncSetAttribute(k_source_disk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  k_source_disk<<<(unsigned)blocks, kSourceThreads, smem, s>>>(mf.as<float2>(), npx, npy, R,
                                                               dt.as<double>(), dfull, out);
  LENS_LAUNCHED("k_source_disk");
  // the host table must outlive the copy
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
