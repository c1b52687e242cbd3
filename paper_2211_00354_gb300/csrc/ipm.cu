// ipm.cu -- first-order Inverse Polygon Mapping (Sec. 2.3; step 4 of the
// FMM-IPM algorithm of Sec. 2.4).  Each image-plane cell (i, j) of a grid
// chunk has corners y[j][i], y[j][i+1], y[j+1][i+1], y[j+1][i]
// (counter-clockwise in the image plane); its source-plane quadrilateral P
// receives the cell area h^2, apportioned over the map pixels by the signed
// overlap fraction a_pix / A_P, and
//     map[pix] += (h^2 / S*) * a_pix / A_P.
//
// Corners arrive in pixel coordinates u = (y1 - u0)/du, v = (y2 - v0)/dv,
// split as (floor, float fraction) by the deflection epilogue, so the common
// case needs no float64 at all:
//   fast path (one thread per cell): pixel bounding box at most 2 x 2 and a
//     well-conditioned polygon -> float32 clipping in coordinates local to
//     the box (a single-pixel box needs no clipping: the fraction is 1);
//   queued path (one warp per cell, lanes striding over the cell's pixels):
//     larger cells in float32, where pixels that no edge meets take the
//     polygon's winding number and only boundary pixels are clipped;
//     ill-conditioned cells (|A_P| small against the box) in float64.
// Overlaps come from a streaming Sutherland-Hodgman chain against the four
// sides of the pixel with a running shoelace sum; clipping against a convex
// window keeps the winding-weighted area, so inverted and self-intersecting
// (critical) cells are handled "naively", as the first-order IPM does.
// Ledger per chunk: area_in_map, area_outside, area_dropped (bbox larger
// than the cap, or a corner beyond 2^30 pixels), area_degenerate
// (|A_P| <= 1e-14 h^2).
#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kIpmThreads = 256;
constexpr int kFar = 0x7fffffff;

// Streaming Sutherland-Hodgman against 4 half-planes (x >= x0, x <= x0+1,
// y >= y0, y <= y0+1) feeding a shoelace accumulator.
template <typename T>
struct ClipChain {
  T bx0, bx1, by0, by1;
  T fx[4], fy[4], px[4], py[4];
  bool pin[4], started[4];
  T ox, oy, lx, ly, area2;
  int nsink;

  __device__ __forceinline__ void init(T x0, T y0) {
    bx0 = x0; bx1 = x0 + (T)1; by0 = y0; by1 = y0 + (T)1;
#pragma unroll
    for (int k = 0; k < 4; ++k) started[k] = false;
    nsink = 0;
    area2 = (T)0;
  }
  __device__ __forceinline__ T val(int K, T x, T y) const {
    switch (K) {
      case 0: return x - bx0;
      case 1: return bx1 - x;
      case 2: return y - by0;
      default: return by1 - y;
    }
  }
  __device__ __forceinline__ void sink(T x, T y) {
    if (nsink == 0) { ox = x; oy = y; }
    else if (nsink >= 2) area2 += (lx - ox) * (y - oy) - (x - ox) * (ly - oy);
    lx = x; ly = y;
    ++nsink;
  }
  template <int K>
  __device__ __forceinline__ void cross_point(T ax, T ay, T va, T cx, T cy, T vc) {
    const T t = va / (va - vc);
    T ix = ax + t * (cx - ax), iy = ay + t * (cy - ay);
    if (K == 0) ix = bx0; else if (K == 1) ix = bx1; else if (K == 2) iy = by0; else iy = by1;
    put<K + 1>(ix, iy);
  }
  template <int K>
  __device__ __forceinline__ void put(T x, T y) {
    if constexpr (K == 4) {
      sink(x, y);
    } else {
      const T v = val(K, x, y);
      const bool in = v >= (T)0;
      if (!started[K]) {
        started[K] = true; fx[K] = x; fy[K] = y;
      } else if (in != pin[K]) {
        cross_point<K>(px[K], py[K], val(K, px[K], py[K]), x, y, v);
      }
      if (in) put<K + 1>(x, y);
      px[K] = x; py[K] = y; pin[K] = in;
    }
  }
  template <int K>
  __device__ __forceinline__ void close() {
    if constexpr (K < 4) {
      if (started[K]) {
        const T vf = val(K, fx[K], fy[K]);
        const bool fin = vf >= (T)0;
        if (fin != pin[K]) cross_point<K>(px[K], py[K], val(K, px[K], py[K]), fx[K], fy[K], vf);
      }
      close<K + 1>();
    }
  }
  __device__ __forceinline__ T area() const { return (T)0.5 * area2; }
};

template <typename T>
__device__ __forceinline__ T overlap(const T* qx, const T* qy, T x0, T y0) {
  ClipChain<T> c;
  c.init(x0, y0);
#pragma unroll
  for (int k = 0; k < 4; ++k) c.template put<0>(qx[k], qy[k]);
  c.template close<0>();
  return c.area();
}

struct IpmArgs {
  const PixCorner* yc;  // (nrows+1) x (nx+1) corners of the chunk
  int64_t nx, ncells;
  double* map;
  double* stats;        // [8]
  int* queue; int* qcount;
  IpmParams ip;
  float thr_area;       // fast-path lower bound on |A_P| in pixel units
};

__device__ __forceinline__ void block_add_stats(double* stats, double in_map, double outside,
                                                double dropped, double degen, double ndrop,
                                                double ndeg, double nupd) {
  __shared__ double sh[7][kIpmThreads / 32];
  double v[7] = {in_map, outside, dropped, degen, ndrop, ndeg, nupd};
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double x = 0;
    for (int q = 0; q < kIpmThreads / 32; ++q) x += sh[threadIdx.x][q];
    if (x != 0.0) atomicAdd(&stats[threadIdx.x + 2], x);
  }
}

__global__ void __launch_bounds__(kIpmThreads) k_ipm_fast(IpmArgs A) {
  const int64_t c = blockIdx.x * (int64_t)kIpmThreads + threadIdx.x;
  double in_map = 0, outside = 0, dropped = 0, degen = 0, ndrop = 0, ndeg = 0, nupd = 0;
  const double ac = A.ip.a_cell;
  if (c < A.ncells) {
    const int64_t j = c / A.nx, i = c - j * A.nx;
    const int64_t W = A.nx + 1;
    PixCorner q4[4];
    q4[0] = A.yc[j * W + i];
    q4[1] = A.yc[j * W + i + 1];
    q4[2] = A.yc[(j + 1) * W + i + 1];
    q4[3] = A.yc[(j + 1) * W + i];
    bool far = false;
    int ix0 = kFar, ix1 = -kFar, iy0 = kFar, iy1 = -kFar;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      far |= (q4[k].iu == kFar) | (q4[k].iv == kFar);
      ix0 = min(ix0, q4[k].iu); ix1 = max(ix1, q4[k].iu);
      iy0 = min(iy0, q4[k].iv); iy1 = max(iy1, q4[k].iv);
    }
    if (far) {
      dropped = ac; ndrop = 1;
    } else if (ix1 < 0 || iy1 < 0 || ix0 > A.ip.npx - 1 || iy0 > A.ip.npy - 1) {
      outside = ac;
    } else if (A.ip.cap > 0 && ((int64_t)ix1 - ix0 + 1 > A.ip.cap || (int64_t)iy1 - iy0 + 1 > A.ip.cap)) {
      dropped = ac; ndrop = 1;
    } else {
      float qx[4], qy[4];
      float xmn = 1e30f, xmx = -1e30f, ymn = 1e30f, ymx = -1e30f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        qx[k] = (float)(q4[k].iu - ix0) + q4[k].fu;
        qy[k] = (float)(q4[k].iv - iy0) + q4[k].fv;
        xmn = fminf(xmn, qx[k]); xmx = fmaxf(xmx, qx[k]);
        ymn = fminf(ymn, qy[k]); ymx = fmaxf(ymx, qy[k]);
      }
      const float A_loc = 0.5f * ((qx[1] - qx[0]) * (qy[2] - qy[0]) - (qx[2] - qx[0]) * (qy[1] - qy[0]) +
                                  (qx[2] - qx[0]) * (qy[3] - qy[0]) - (qx[3] - qx[0]) * (qy[2] - qy[0]));
      const float ext = (xmx - xmn) * (ymx - ymn);
      const bool small = (ix1 - ix0 <= 1) && (iy1 - iy0 <= 1);
      const bool good = fabsf(A_loc) > 1e-3f * ext && fabsf(A_loc) > A.thr_area;
      if (small && good) {
        if (ix0 == ix1 && iy0 == iy1) {
          atomicAdd(&A.map[(int64_t)iy0 * A.ip.npx + ix0], A.ip.scale);
          in_map = ac;
          nupd = 1;
        } else {
          const float inv = 1.0f / A_loc;
          double fin = 0.0;
          for (int py = iy0; py <= iy1; ++py) {
            if (py < 0 || py >= A.ip.npy) continue;
            for (int px = ix0; px <= ix1; ++px) {
              if (px < 0 || px >= A.ip.npx) continue;
              const float a = overlap<float>(qx, qy, (float)(px - ix0), (float)(py - iy0));
              if (a == 0.0f) continue;
              const float fr = a * inv;
              atomicAdd(&A.map[(int64_t)py * A.ip.npx + px], A.ip.scale * (double)fr);
              fin += (double)fr;
              nupd += 1;
            }
          }
          in_map = ac * fin;
          outside = ac * (1.0 - fin);
        }
      } else {
        const int slot = atomicAdd(A.qcount, 1);
        A.queue[slot] = (int)c;
      }
    }
  }
  block_add_stats(A.stats, in_map, outside, dropped, degen, ndrop, ndeg, nupd);
}

// Does the segment P->Q meet the closed unit square at (ox, oy)?
__device__ __forceinline__ bool seg_meets_pixel(float px, float py, float qx, float qy, float ox,
                                                float oy) {
  if (fmaxf(px, qx) < ox || fminf(px, qx) > ox + 1.f || fmaxf(py, qy) < oy ||
      fminf(py, qy) > oy + 1.f)
    return false;
  const float dx = qx - px, dy = qy - py;
  const float c00 = dx * (oy - py) - dy * (ox - px);
  const float c10 = c00 - dy, c01 = c00 + dx, c11 = c00 + dx - dy;
  const float lo = fminf(fminf(c00, c10), fminf(c01, c11));
  const float hi = fmaxf(fmaxf(c00, c10), fmaxf(c01, c11));
  return !(lo > 0.f || hi < 0.f);
}

// winding number of the closed polygon q around (x, y)
__device__ __forceinline__ int winding4(const float* qx, const float* qy, float x, float y) {
  int w = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float ax = qx[e], ay = qy[e], bx = qx[(e + 1) & 3], by = qy[(e + 1) & 3];
    const float cr = (bx - ax) * (y - ay) - (x - ax) * (by - ay);
    if (ay <= y && by > y && cr > 0.f) ++w;
    else if (by <= y && ay > y && cr < 0.f) --w;
  }
  return w;
}

// One warp per queued cell (bounding box larger than 2 x 2 pixels, or an
// ill-conditioned polygon).  Well-conditioned cells run in float32 in
// coordinates local to their box: a pixel that no edge meets is covered by
// the polygon's winding number exactly, so only pixels on the boundary are
// clipped.  Ill-conditioned cells (|A_P| small against the box) run the full
// clip in float64.
__global__ void __launch_bounds__(kIpmThreads) k_ipm_queue(IpmArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t wg = (blockIdx.x * (int64_t)kIpmThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kIpmThreads) >> 5;
  const int nq = *A.qcount;
  const double ac = A.ip.a_cell;
  double in_map = 0, outside = 0, degen = 0, ndeg = 0, nupd = 0;
  for (int64_t t = wg; t < nq; t += nwarps) {
    const int64_t c = A.queue[t];
    const int64_t j = c / A.nx, i = c - j * A.nx;
    const int64_t W = A.nx + 1;
    PixCorner q4[4];
    q4[0] = A.yc[j * W + i];
    q4[1] = A.yc[j * W + i + 1];
    q4[2] = A.yc[(j + 1) * W + i + 1];
    q4[3] = A.yc[(j + 1) * W + i];
    int ix0 = kFar, ix1 = -kFar, iy0 = kFar, iy1 = -kFar;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ix0 = min(ix0, q4[k].iu); ix1 = max(ix1, q4[k].iu);
      iy0 = min(iy0, q4[k].iv); iy1 = max(iy1, q4[k].iv);
    }
    const int cx0 = max(ix0, 0), cx1 = min(ix1, A.ip.npx - 1);
    const int cy0 = max(iy0, 0), cy1 = min(iy1, A.ip.npy - 1);
    const int64_t w = (int64_t)cx1 - cx0 + 1, npix = w * ((int64_t)cy1 - cy0 + 1);
    float fx[4], fy[4];
    float xmn = 1e30f, xmx = -1e30f, ymn = 1e30f, ymx = -1e30f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      fx[k] = (float)(q4[k].iu - ix0) + q4[k].fu;
      fy[k] = (float)(q4[k].iv - iy0) + q4[k].fv;
      xmn = fminf(xmn, fx[k]); xmx = fmaxf(xmx, fx[k]);
      ymn = fminf(ymn, fy[k]); ymx = fmaxf(ymx, fy[k]);
    }
    const float A_loc = 0.5f * ((fx[1] - fx[0]) * (fy[2] - fy[0]) - (fx[2] - fx[0]) * (fy[1] - fy[0]) +
                                (fx[2] - fx[0]) * (fy[3] - fy[0]) - (fx[3] - fx[0]) * (fy[2] - fy[0]));
    const bool fp32 = fabsf(A_loc) > 2e-2f * (xmx - xmn) * (ymx - ymn) && fabsf(A_loc) > A.thr_area;
    double fin = 0.0;
    if (fp32) {
      const float inv = 1.0f / A_loc;
      for (int64_t t2 = lane; t2 < npix; t2 += 32) {
        const int py = cy0 + (int)(t2 / w), px = cx0 + (int)(t2 % w);
        const float ox = (float)(px - ix0), oy = (float)(py - iy0);
        bool cut = false;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          cut |= seg_meets_pixel(fx[e], fy[e], fx[(e + 1) & 3], fy[(e + 1) & 3], ox, oy);
        const float a = cut ? overlap<float>(fx, fy, ox, oy)
                            : (float)winding4(fx, fy, ox + 0.5f, oy + 0.5f);
        if (a == 0.0f) continue;
        const float fr = a * inv;
        atomicAdd(&A.map[(int64_t)py * A.ip.npx + px], A.ip.scale * (double)fr);
        fin += (double)fr;
        nupd += 1;
      }
    } else {
      double u[4], v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        u[k] = (double)q4[k].iu + (double)q4[k].fu;
        v[k] = (double)q4[k].iv + (double)q4[k].fv;
      }
      const double A_P = 0.5 * ((u[1] - u[0]) * (v[2] - v[0]) - (u[2] - u[0]) * (v[1] - v[0]) +
                                (u[2] - u[0]) * (v[3] - v[0]) - (u[3] - u[0]) * (v[2] - v[0]));
      if (!(fabs(A_P) * A.ip.s_star > 1e-14 * ac)) {
        if (lane == 0) { degen += ac; ndeg += 1; }
        continue;
      }
      const double inv = 1.0 / A_P;
      for (int64_t t2 = lane; t2 < npix; t2 += 32) {
        const int64_t py = cy0 + t2 / w, px = cx0 + t2 % w;
        double qx[4], qy[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { qx[k] = u[k] - (double)px; qy[k] = v[k] - (double)py; }
        const double a = overlap<double>(qx, qy, 0.0, 0.0);
        if (a == 0.0) continue;
        const double fr = a * inv;
        atomicAdd(&A.map[py * A.ip.npx + px], A.ip.scale * fr);
        fin += fr;
        nupd += 1;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fin += __shfl_xor_sync(0xffffffffu, fin, o);
    if (lane == 0) { in_map += ac * fin; outside += ac * (1.0 - fin); }
  }
  block_add_stats(A.stats, in_map, outside, 0.0, degen, 0.0, ndeg, nupd);
}

}  // namespace

std::pair<cudaEvent_t, cudaEvent_t> event_pair_begin(cudaStream_t s) {
  std::pair<cudaEvent_t, cudaEvent_t> e;
  LENS_CUDA(cudaEventCreate(&e.first));
  LENS_CUDA(cudaEventCreate(&e.second));
  LENS_CUDA(cudaEventRecord(e.first, s));
  return e;
}
void event_pair_end(std::pair<cudaEvent_t, cudaEvent_t>& e, cudaStream_t s) {
  LENS_CUDA(cudaEventRecord(e.second, s));
}

void ipm_accumulate(const PixCorner* yc, int64_t nx, int64_t nrows_cells, const IpmParams& ip,
                    double* map, double* stats_dev, int* queue, int* qcount, cudaStream_t s,
                    std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev) {
  const int64_t ncells = nx * nrows_cells;
  if (ncells <= 0) return;
  IpmArgs A{};
  A.yc = yc; A.nx = nx; A.ncells = ncells; A.map = map; A.stats = stats_dev;
  A.queue = queue; A.qcount = qcount; A.ip = ip;
  A.thr_area = (float)(1e-13 * ip.a_cell / ip.s_star);
  LENS_CUDA(cudaMemsetAsync(qcount, 0, sizeof(int), s));
  std::pair<cudaEvent_t, cudaEvent_t> e;
  if (ev) e = event_pair_begin(s);
  k_ipm_fast<<<grid_for(ncells, kIpmThreads), kIpmThreads, 0, s>>>(A);
  LENS_LAUNCHED("k_ipm_fast");
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  k_ipm_queue<<<sms * 8, kIpmThreads, 0, s>>>(A);
  LENS_LAUNCHED("k_ipm_queue");
  if (ev) {
    event_pair_end(e, s);
    ev->push_back(e);
  }
}

}  // namespace lens
