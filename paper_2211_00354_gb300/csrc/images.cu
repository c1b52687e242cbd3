// images.cu -- images of a point source and the lensed image of a Gaussian
// source on a deflected ray grid (Sec. 2.5: the images of a background
// Gaussian source behind a simulated halo, found from the deflections of a
// regular ray grid).
//  * find_images: thread per cell.  A cell holds an image of beta when beta
//    lies in the bounding box of its four deflected corners and their closed
//    polygon (i,j) -> (i+1,j) -> (i+1,j+1) -> (i,j+1) winds around beta (the
//    cell polygons of the IPM, Sec. 2.3).  The crossing rule takes half-open
//    edge spans in y, and each orientation product is rounded float64
//    without contraction, so a source on an edge shared by two cells is
//    claimed by the same cell on any machine.  Inside an image cell the
//    corners' bilinear interpolation is inverted by 20 Newton steps from the
//    cell centre (cell coordinates kept within [-1, 2]); the image is that
//    point, its signed magnification h^2 / det J of the bilinear map there.
//    Image cells are few: each takes a slot from one counter.  The float64
//    pipe is GB300's slowest, so every cell first passes an integer test on
//    the high words of its corner coordinates (a key that never decreases
//    with the value, one unit of slack for -0/+0): only the cells whose
//    coarse bounding box can hold beta reach the float64 test above.
//  * source_image: exp(-|y - beta|^2 / 2 sigma^2) per ray (lensing keeps
//    surface brightness).
#include "cx.cuh"
#include "images.h"

namespace lens {
namespace {

constexpr int kNewtonSteps = 20;

__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// sign, exponent and top 20 mantissa bits of v as an int that never
// decreases when v increases (-0 sits one below +0)
__device__ __forceinline__ int okey(double v) {
  const int h = __double2hiint(v);
  return h ^ ((h >> 31) & 0x7fffffff);
}

// (b - a) x (p - a), each product and difference rounded once
__device__ __forceinline__ double orient(double2 a, double2 b, double px, double py) {
  return __dsub_rn(__dmul_rn(__dsub_rn(b.x, a.x), __dsub_rn(py, a.y)),
                   __dmul_rn(__dsub_rn(px, a.x), __dsub_rn(b.y, a.y)));
}

__global__ void k_find_images(const double2* __restrict__ y, int64_t nx, int64_t ny, double b1,
                              double b2, double x0, double y0, double h, int64_t max_out,
                              unsigned long long* __restrict__ count, double* __restrict__ out,
                              int64_t* __restrict__ cells) {
  const int64_t n = nx * ny, W = nx + 1;
  const bool small = n < (1ll << 32);
  const int kb1 = okey(b1), kb2 = okey(b2);  // beta finite: no overflow below
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = small ? (int64_t)((uint32_t)c / (uint32_t)nx) : c / nx, i = c - j * nx;
    const double2 q[4] = {y[j * W + i], y[j * W + i + 1], y[(j + 1) * W + i + 1], y[(j + 1) * W + i]};
    int kx0 = okey(q[0].x), kx1 = kx0, ky0 = okey(q[0].y), ky1 = ky0;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      const int kx = okey(q[k].x), ky = okey(q[k].y);
      kx0 = min(kx0, kx); kx1 = max(kx1, kx);
      ky0 = min(ky0, ky); ky1 = max(ky1, ky);
    }
    // necessary for the exact test: x <= b implies okey(x) <= okey(b) + 1
    if (kx0 > kb1 + 1 || kx1 < kb1 - 1 || ky0 > kb2 + 1 || ky1 < kb2 - 1) continue;
    // a NaN corner leaves the bounding box undefined: no image (fmin and
    // fmax would drop the NaN operand and build the box from the others)
    bool nan = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) nan |= isnan(q[k].x) | isnan(q[k].y);
    if (nan) continue;
    double xmn = q[0].x, xmx = q[0].x, ymn = q[0].y, ymx = q[0].y;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      xmn = fmin(xmn, q[k].x); xmx = fmax(xmx, q[k].x);
      ymn = fmin(ymn, q[k].y); ymx = fmax(ymx, q[k].y);
    }
    if (!(xmn <= b1 && b1 <= xmx && ymn <= b2 && b2 <= ymx)) continue;
    int w = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const double2 a = q[e], b = q[(e + 1) & 3];
      const double cr = orient(a, b, b1, b2);
      if (a.y <= b2 && b2 < b.y && cr > 0.0) ++w;
      else if (b.y <= b2 && b2 < a.y && cr < 0.0) --w;
    }
    if (w == 0) continue;
    // p(s, t) = q0 + s e + t f + s t g
    const double2 e = sub2(q[1], q[0]), f = sub2(q[3], q[0]);
    const double2 g = sub2(make_double2(q[0].x - q[1].x + q[2].x, q[0].y - q[1].y + q[2].y), q[3]);
    double s = 0.5, t = 0.5;
    for (int it = 0; it < kNewtonSteps; ++it) {
      const double2 js = make_double2(e.x + t * g.x, e.y + t * g.y);
      const double2 jt = make_double2(f.x + s * g.x, f.y + s * g.y);
      const double st = s * t;
      const double rx = b1 - (q[0].x + s * e.x + t * f.x + st * g.x);
      const double ry = b2 - (q[0].y + s * e.y + t * f.y + st * g.y);
      const double det = js.x * jt.y - jt.x * js.y;
      if (det == 0.0) break;
      const double ds = (rx * jt.y - jt.x * ry) / det, dt = (js.x * ry - rx * js.y) / det;
      s = fmin(fmax(s + ds, -1.0), 2.0);
      t = fmin(fmax(t + dt, -1.0), 2.0);
    }
    const double2 js = make_double2(e.x + t * g.x, e.y + t * g.y);
    const double2 jt = make_double2(f.x + s * g.x, f.y + s * g.y);
    const double det = js.x * jt.y - jt.x * js.y;
    const unsigned long long slot = atomicAdd(count, 1ull);
    if (slot < (unsigned long long)max_out) {
      out[3 * slot + 0] = x0 + ((double)i + s) * h;
      out[3 * slot + 1] = y0 + ((double)j + t) * h;
      out[3 * slot + 2] = det != 0.0 ? h * h / det : INFINITY;
      cells[slot] = c;
    }
  }
}

// exp(-q / 2 sigma^2) per ray; beyond q = 746 * 2 sigma^2 the float64 value
// is 0 (e^-746 is below half the least subnormal), so the division and the
// exponential run only for the rays near the source -- on a whole map a
// small share, and each costs some 30 operations of GB300's slow float64 pipe
__global__ void k_source_image(const double2* __restrict__ y, int64_t m, double b1, double b2,
                               double two_s2, double qmax, double* __restrict__ out) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const double dx = y[r].x - b1, dy = y[r].y - b2;
  const double q = dx * dx + dy * dy;
  out[r] = q > qmax ? 0.0 : exp(-q / two_s2);
}

}  // namespace

int64_t find_images(const double* y, int64_t nx, int64_t ny, double x0, double y0, double h,
                    double b1, double b2, int64_t max_out, double* out, int64_t* cells,
                    DeviceAlloc& da, cudaStream_t s) {
  Scratch dcount(&da, sizeof(unsigned long long));
  LENS_CUDA(cudaMemsetAsync(dcount.p, 0, sizeof(unsigned long long), s));
  const int64_t n = nx * ny;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32);
  k_find_images<<<blocks, 256, 0, s>>>(reinterpret_cast<const double2*>(y), nx, ny, b1, b2, x0,
                                        y0, h, max_out, dcount.as<unsigned long long>(), out, cells);
  LENS_LAUNCHED("k_find_images");
  unsigned long long found = 0;
  LENS_CUDA(cudaMemcpyAsync(&found, dcount.p, sizeof(found), cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaStreamSynchronize(s));
  return (int64_t)found;
}

void source_image(const double* y, int64_t m, double b1, double b2, double sigma, double* out,
                  cudaStream_t s) {
  if (m == 0) return;
  k_source_image<<<grid_for(m, 256), 256, 0, s>>>(reinterpret_cast<const double2*>(y), m, b1, b2,
                                                  2.0 * sigma * sigma, 746.0 * 2.0 * sigma * sigma,
                                                  out);
  LENS_LAUNCHED("k_source_image");
}

}  // namespace lens
