// multiplane.cu -- rays through several thin lens planes (Sec. 1: ray
// tracing through several lens planes repeats the mapping plane by plane; a
// thick lens is a collection of thin planes).  Plane i (in order of distance)
// holds point lenses and a smooth field; with each deflection scaled to the
// source plane as in Eq. 1,
//     alpha_i(x) = sum_k m_ik (x - x_ik) / |x - x_ik|^2
//                  + diag(kappa_i + gamma_i, kappa_i - gamma_i) x,
// a ray entering at x_1 reaches plane j at
//     x_j = x_1 - sum_{i<j} beta_ij alpha_i(x_i)
// and the source plane at y = x_1 - sum_i alpha_i(x_i).
//
// Per plane: the bounding box of the rays' positions x_i (one reduction,
// read back), an FMM plan over the plane's stars with that box as its target
// region (the star sum only: the smooth field is added here exactly), the
// plan's deflection of the rays (the same kernels as lens_deflect), then one
// kernel that forms alpha_i = x_i - y_i + diag(...) x_i, keeps it, and moves
// every ray on to the next plane (or to the source plane after the last).
// lens_multiplane_ipm_map runs the chunk loop of Sec. 2.4 with these
// positions: each chunk's corner rays are traced through all planes, turned
// into pixel coordinates and apportioned by the same IPM kernels as
// lens_ipm_map.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lens_internal.h"
#include "okey.cuh"

namespace lens {
namespace {

constexpr int kMaxPlanes = 64;
constexpr int kBoundsBlocks = 256;
constexpr int kFarPix = 0x7fffffff;

// per block: min/max of x and y over its share of the points, and whether
// any coordinate is not finite
// the bounding box of m positions by order-preserving integer keys of the
// float64 values (okey.cuh: exact, on the integer pipe), one partial box per
// block

__global__ void k_mp_bounds(const double2* __restrict__ x, int64_t m, double* __restrict__ part,
                            int* __restrict__ bad) {
  __shared__ unsigned long long sh[4][8];
  unsigned long long x0 = ~0ull, x1 = 0ull, y0 = ~0ull, y1 = 0ull;
  int nf = 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double2 p = x[r];
    if (!(finite_bits(p.x) && finite_bits(p.y))) { nf = 1; continue; }
    const unsigned long long kx = okey(p.x), ky = okey(p.y);
    x0 = min(x0, kx); x1 = max(x1, kx);
    y0 = min(y0, ky); y1 = max(y1, ky);
  }
  if (__any_sync(0xffffffffu, nf) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x0 = min(x0, __shfl_xor_sync(0xffffffffu, x0, o)); x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, o));
    y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, o)); y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, o));
  }
  const int t = threadIdx.x, w = t >> 5;
  if ((t & 31) == 0) { sh[0][w] = x0; sh[1][w] = x1; sh[2][w] = y0; sh[3][w] = y1; }
  __syncthreads();
  if (t < 4) {
    unsigned long long v = sh[t][0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) v = (t & 1) ? max(v, sh[t][q]) : min(v, sh[t][q]);
    // an empty block keeps +inf / -inf, as the float64 form did
    part[4 * blockIdx.x + t] = (t & 1) ? (v == 0ull ? -INFINITY : unkey(v))
                                       : (v == ~0ull ? INFINITY : unkey(v));
  }
}

struct MpStep {
  const double2* x1;  // entry points x_1
  const double2* xi;  // positions at plane i
  const double2* yi;  // x_i mapped by plane i's stars alone (x - star sum), or NULL (no stars)
  double2* alpha;     // K x m: alpha_k of the planes done so far
  double2* xnext;     // positions at plane i+1, or y after the last plane
  double2* xsave;     // copy of xnext for the caller (NULL: none)
  double kg1, kg2;    // kappa_i + gamma_i, kappa_i - gamma_i
  double w[kMaxPlanes];  // w[k] = beta_{k, i+1} for k <= i (1 for the source plane)
  int i;
  int64_t m;
};

// alpha_i at every ray, then x_{i+1} = x_1 - sum_{k<=i} w_k alpha_k (summed
// in plane order)
__global__ void k_mp_step(MpStep A) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= A.m) return;
  const double2 x = A.xi[r];
  double a1 = A.kg1 * x.x, a2 = A.kg2 * x.y;
  if (A.yi) {
    const double2 y = A.yi[r];
    a1 += x.x - y.x;
    a2 += x.y - y.y;
  }
  A.alpha[(int64_t)A.i * A.m + r] = make_double2(a1, a2);
  double s1 = 0.0, s2 = 0.0;
  for (int k = 0; k < A.i; ++k) {
    const double2 ak = A.alpha[(int64_t)k * A.m + r];
    s1 += A.w[k] * ak.x;
    s2 += A.w[k] * ak.y;
  }
  s1 += A.w[A.i] * a1;
  s2 += A.w[A.i] * a2;
  const double2 x1 = A.x1[r];
  const double2 xn = make_double2(x1.x - s1, x1.y - s2);
  A.xnext[r] = xn;
  if (A.xsave) A.xsave[r] = xn;
}

// corner rays of grid rows row0 .. row0 + nrows - 1: x0 + i h, y0 + j h
// (one rounding per product and sum, as the grid defines them)
__global__ void k_mp_grid_rays(double x0, double y0, double h, int64_t nx1, int64_t row0,
                               int64_t n, double2* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t j = t / nx1, i = t - j * nx1;
  out[t] = make_double2(__dadd_rn(x0, __dmul_rn((double)i, h)),
                        __dadd_rn(y0, __dmul_rn((double)(row0 + j), h)));
}

// source-plane positions -> pixel coordinates (integer pixel + float32
// fraction), corners beyond 2^30 pixels marked far
__global__ void k_mp_pix(const double2* __restrict__ y, int64_t n, IpmParams ip,
                         PixCorner* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double2 p = y[t];
  const double u = (p.x - ip.u0) * ip.inv_du, v = (p.y - ip.v0) * ip.inv_dv;
  PixCorner pc;
  if (!(fabs(u) < 5.0e8) || !(fabs(v) < 5.0e8)) {
    pc.iu = kFarPix; pc.fu = 0.f; pc.iv = kFarPix; pc.fv = 0.f;
  } else {
    const double fu = floor(u), fv = floor(v);
    pc.iu = (int)fu; pc.fu = (float)(u - fu);
    pc.iv = (int)fv; pc.fv = (float)(v - fv);
    if (pc.fu >= 1.f) { pc.iu += 1; pc.fu = 0.f; }
    if (pc.fv >= 1.f) { pc.iv += 1; pc.fv = 0.f; }
  }
  out[t] = pc;
}

struct PlaneSet {
  const lens_plane* planes;
  int K;
  const double* beta;  // host K x K
  lens_build_opts opts;
  const lens_allocator* allocator;
};

void check_planes(const PlaneSet& ps) {
  if (ps.K < 1 || ps.K > kMaxPlanes) fail(LENS_EINVAL, "the number of planes must be in 1..64");
  if (!ps.planes || !ps.beta) fail(LENS_EINVAL, "planes or beta is NULL");
  for (int i = 0; i < ps.K; ++i) {
    const lens_plane& p = ps.planes[i];
    if (p.n < 0 || p.n >= (int64_t)INT32_MAX) fail(LENS_EINVAL, "a plane's star count is out of range");
    if (p.n > 0 && (!p.stars_xy || !p.masses)) fail(LENS_EINVAL, "a plane's stars or masses is NULL");
    if (!std::isfinite(p.kappa_s) || !std::isfinite(p.gamma))
      fail(LENS_EINVAL, "a plane's kappa_s and gamma must be finite");
    for (int j = i + 1; j < ps.K; ++j)
      if (!std::isfinite(ps.beta[i * ps.K + j])) fail(LENS_EINVAL, "beta must be finite");
  }
}

// bounding box of m positions; LENS_EDOMAIN if any is not finite
void bounds(const double2* x, int64_t m, double box[4], DeviceAlloc& da, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(kBoundsBlocks, (m + 255) / 256);
  Scratch part(&da, sizeof(double) * 4 * blocks + sizeof(int) * 4);
  int* bad = reinterpret_cast<int*>(part.as<double>() + 4 * blocks);
  LENS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  k_mp_bounds<<<blocks, 256, 0, s>>>(x, m, part.as<double>(), bad);
  LENS_LAUNCHED("k_mp_bounds");
  std::vector<double> h(4 * (size_t)blocks + 2);
  LENS_CUDA(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * 4 * blocks + sizeof(int),
                            cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaStreamSynchronize(s));
  int nb = 0;
  std::memcpy(&nb, h.data() + 4 * blocks, sizeof(int));
  if (nb) fail(LENS_EDOMAIN, "a ray position is not finite");
  box[0] = box[2] = INFINITY;
  box[1] = box[3] = -INFINITY;
  for (int b = 0; b < blocks; ++b) {
    box[0] = std::min(box[0], h[4 * b]); box[1] = std::max(box[1], h[4 * b + 1]);
    box[2] = std::min(box[2], h[4 * b + 2]); box[3] = std::max(box[3], h[4 * b + 3]);
  }
}

// Trace m rays x1 through every plane: y (m x 2) and, if xsave is given, the
// positions at each plane (K x m x 2).  Returns the stars' work in rays
// deflected (m per plane with stars).
int64_t trace(const PlaneSet& ps, const double2* x1, int64_t m, double2* y, double2* xsave,
              DeviceAlloc& da, cudaStream_t s) {
  const int K = ps.K;
  Scratch alpha(&da, sizeof(double2) * (size_t)K * (size_t)m);
  Scratch xa(&da, sizeof(double2) * (size_t)m), xb(&da, sizeof(double2) * (size_t)m);
  Scratch yi(&da, sizeof(double2) * (size_t)m);
  if (xsave)
    LENS_CUDA(cudaMemcpyAsync(xsave, x1, sizeof(double2) * (size_t)m, cudaMemcpyDeviceToDevice, s));
  const double2* xi = x1;
  int64_t work = 0;
  for (int i = 0; i < K; ++i) {
    const lens_plane& pl = ps.planes[i];
    bool stars = pl.n > 0;
    if (stars) {
      lens_build_opts o = ps.opts;
      o.has_target_box = 1;
      bounds(xi, m, o.target_box, da, s);
      lens_plan* plan = nullptr;
      lens_status st = lens_fmm_build(pl.stars_xy, pl.masses, pl.n, 0.0, 0.0, &o, ps.allocator,
                                      (void*)s, &plan);
      if (st != LENS_OK) fail(st, std::string("plane ") + std::to_string(i) + ": " + lens_last_error());
      st = lens_deflect(plan, reinterpret_cast<const double*>(xi), m, yi.as<double>(), nullptr,
                        (void*)s);
      const std::string msg = st == LENS_OK ? "" : lens_last_error();
      lens_plan_destroy(plan);
      if (st != LENS_OK) fail(st, std::string("plane ") + std::to_string(i) + ": " + msg);
      work += m;
    }
    MpStep A{};
    A.x1 = x1; A.xi = xi; A.yi = stars ? yi.as<double2>() : nullptr;
    A.alpha = alpha.as<double2>();
    const bool last = i == K - 1;
    double2* xn = last ? y : (i % 2 == 0 ? xa.as<double2>() : xb.as<double2>());
    A.xnext = xn;
    A.xsave = (!last && xsave) ? xsave + (size_t)(i + 1) * (size_t)m : nullptr;
    A.kg1 = pl.kappa_s + pl.gamma;
    A.kg2 = pl.kappa_s - pl.gamma;
    for (int k = 0; k <= i; ++k) A.w[k] = last ? 1.0 : ps.beta[k * K + (i + 1)];
    A.i = i;
    A.m = m;
    k_mp_step<<<grid_for(m, 256), 256, 0, s>>>(A);
    LENS_LAUNCHED("k_mp_step");
    xi = xn;
  }
  return work;
}

}  // namespace
}  // namespace lens

using namespace lens;

extern "C" lens_status lens_multiplane_deflect(const lens_plane* planes, int nplanes,
                                               const double* beta, const lens_build_opts* opts,
                                               const double* rays_xy, int64_t m, double* y_out,
                                               double* x_planes_out,
                                               const lens_allocator* allocator, void* stream) {
  try {
    if (!opts) fail(LENS_EINVAL, "opts is NULL");
    PlaneSet ps{planes, nplanes, beta, *opts, allocator};
    check_planes(ps);
    if (m < 0) fail(LENS_EINVAL, "m must be >= 0");
    if (m > 0 && (!rays_xy || !y_out)) fail(LENS_EINVAL, "rays or y_out is NULL");
    if (m >= (int64_t)INT32_MAX) fail(LENS_EINVAL, "too many rays in one call");
    if (m > 0) {
      cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
      DeviceAlloc da;
      da.stream = s;
      if (allocator && allocator->alloc && allocator->free) { da.a = *allocator; da.custom = true; }
      trace(ps, reinterpret_cast<const double2*>(rays_xy), m, reinterpret_cast<double2*>(y_out),
            reinterpret_cast<double2*>(x_planes_out), da, s);
    }
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    set_last_error(std::string("internal: ") + e.what());
    return LENS_ECUDA;
  }
  set_last_error("");
  return LENS_OK;
}

extern "C" lens_status lens_multiplane_ipm_map(const lens_plane* planes, int nplanes,
                                               const double* beta, const lens_build_opts* opts,
                                               const lens_grid* grid, const lens_box* box, int npx,
                                               int npy, int64_t max_cells_per_chunk,
                                               int bbox_cap_px, double* map_out,
                                               lens_ipm_stats* stats,
                                               const lens_allocator* allocator, void* stream) {
  try {
    if (!opts) fail(LENS_EINVAL, "opts is NULL");
    PlaneSet ps{planes, nplanes, beta, *opts, allocator};
    check_planes(ps);
    if (!grid || !box || !map_out) fail(LENS_EINVAL, "grid, box or map_out is NULL");
    if (!(std::isfinite(grid->x0) && std::isfinite(grid->y0) && std::isfinite(grid->h) && grid->h > 0))
      fail(LENS_EINVAL, "grid x0, y0 must be finite and h > 0");
    if (grid->nx < 1 || grid->ny < 1 || grid->nx >= (1ll << 30))
      fail(LENS_EINVAL, "grid needs 1 <= nx < 2^30 and ny >= 1");
    if (!(npx >= 1 && npy >= 1 && (int64_t)npx * npy < (1ll << 31)))
      fail(LENS_EINVAL, "npx, npy must be >= 1 with npx*npy < 2^31");
    if (!(std::isfinite(box->u0) && std::isfinite(box->u1) && std::isfinite(box->v0) &&
          std::isfinite(box->v1) && box->u1 > box->u0 && box->v1 > box->v0))
      fail(LENS_EINVAL, "map window must be finite with u1 > u0, v1 > v0");
    if (max_cells_per_chunk < 0 || bbox_cap_px < 0) fail(LENS_EINVAL, "chunk size and cap must be >= 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceAlloc da;
    da.stream = s;
    if (allocator && allocator->alloc && allocator->free) { da.a = *allocator; da.custom = true; }
    const int64_t nx = grid->nx, ny = grid->ny;
    int64_t max_cells = max_cells_per_chunk;
    if (max_cells == 0) {
      size_t fr = 0, tot = 0;
      LENS_CUDA(cudaMemGetInfo(&fr, &tot));
      // per corner: entry, two positions, plane output, K deflections, the
      // pixel corner; within a quarter of free memory
      const double per = 16.0 * (4 + ps.K) + 16.0 + 4.0;
      max_cells = (int64_t)std::min<double>((double)fr / 4.0 / per, (double)(1ll << 30));
    }
    constexpr int64_t kFlushCellsPerPixel = 64;
    const int64_t flush_cells = std::min<int64_t>(kFlushCellsPerPixel * npx * npy, 1ll << 30);
    max_cells = std::min(std::min<int64_t>(max_cells, 1ll << 30), flush_cells);
    int64_t rows = std::min<int64_t>(std::max<int64_t>(1, max_cells / nx), ny);
    if (!(rows * nx <= (1ll << 30) || rows == 1)) fail(LENS_EINVAL, "grid rows too wide for one chunk");
    if ((rows + 1) * (nx + 1) >= (int64_t)INT32_MAX) rows = std::max<int64_t>(1, (int64_t)INT32_MAX / (nx + 1) - 2);

    IpmParams ip{};
    const double du = (box->u1 - box->u0) / npx, dv = (box->v1 - box->v0) / npy;
    ip.u0 = box->u0; ip.v0 = box->v0;
    ip.inv_du = 1.0 / du; ip.inv_dv = 1.0 / dv;
    ip.a_cell = grid->h * grid->h;
    ip.s_star = du * dv;
    ip.scale = ip.a_cell / ip.s_star;
    ip.npx = npx; ip.npy = npy; ip.cap = bbox_cap_px;

    const size_t ncorn = (size_t)(rows + 1) * (size_t)(nx + 1);
    Scratch rays(&da, sizeof(double2) * ncorn), ys(&da, sizeof(double2) * ncorn);
    Scratch corners(&da, sizeof(PixCorner) * ncorn);
    Scratch queue(&da, sizeof(int) * (size_t)rows * (size_t)nx + sizeof(int) * 4);
    Scratch sdev(&da, sizeof(double) * 16);
    Scratch map32(&da, sizeof(float) * (size_t)npx * (size_t)npy);
    Scratch rowdiff(&da, sizeof(float) * ((size_t)npx + 1) * (size_t)npy);
    int* qcount = queue.as<int>() + (size_t)rows * (size_t)nx;
    LENS_CUDA(cudaMemsetAsync(map32.p, 0, map32.bytes, s));
    LENS_CUDA(cudaMemsetAsync(rowdiff.p, 0, rowdiff.bytes, s));
    LENS_CUDA(cudaMemsetAsync(sdev.p, 0, sdev.bytes, s));
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    struct Clear {
      std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& e;
      ~Clear() { for (auto& p : e) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); } }
    } clear{ev};
    const long long l0 = launch_count();
    int64_t chunks = 0, pending = 0, traced = 0;
    bool flushed = false;
    for (int64_t r0 = 0; r0 < ny; r0 += rows) {
      const int64_t nr = std::min<int64_t>(rows, ny - r0);
      if (pending > 0 && pending + nr * nx > flush_cells) {
        ipm_finish_map(map32.as<float>(), rowdiff.as<float>(), npx, npy, map_out, flushed, true, s);
        flushed = true;
        pending = 0;
      }
      const int64_t nc = (nr + 1) * (nx + 1);
      k_mp_grid_rays<<<grid_for(nc, 256), 256, 0, s>>>(grid->x0, grid->y0, grid->h, nx + 1, r0, nc,
                                                        rays.as<double2>());
      LENS_LAUNCHED("k_mp_grid_rays");
      traced += trace(ps, rays.as<double2>(), nc, ys.as<double2>(), nullptr, da, s);
      k_mp_pix<<<grid_for(nc, 256), 256, 0, s>>>(ys.as<double2>(), nc, ip, corners.as<PixCorner>());
      LENS_LAUNCHED("k_mp_pix");
      ipm_accumulate(corners.as<PixCorner>(), nx, nr, ip, map32.as<float>(), rowdiff.as<float>(),
                     sdev.as<double>(), queue.as<int>(), qcount, nullptr, nullptr, s, &ev);
      pending += nr * nx;
      ++chunks;
    }
    ipm_finish_map(map32.as<float>(), rowdiff.as<float>(), npx, npy, map_out, flushed, false, s);
    double hs[16];
    LENS_CUDA(cudaMemcpyAsync(hs, sdev.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
    LENS_CUDA(cudaStreamSynchronize(s));
    double msk = 0;
    for (auto& e : ev) { float ms = 0; cudaEventElapsedTime(&ms, e.first, e.second); msk += ms; }
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      stats->cells = (double)nx * (double)ny;
      stats->area_total = stats->cells * ip.a_cell;
      stats->area_in_map = ip.a_cell * hs[2];
      stats->area_outside = ip.a_cell * hs[3];
      stats->area_dropped = ip.a_cell * hs[6];
      stats->area_degenerate = ip.a_cell * hs[7];
      stats->cells_dropped = hs[4];
      stats->cells_degenerate = hs[5];
      stats->chunks = chunks;
      stats->rays = (double)traced;
      stats->ipm_updates = hs[8];
      stats->cells_queued = hs[9];
      stats->cells_ext = hs[10];
      stats->ms_ipm_kernel = msk;
      stats->launches = launch_count() - l0;
    }
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    set_last_error(std::string("internal: ") + e.what());
    return LENS_ECUDA;
  }
  set_last_error("");
  return LENS_OK;
}
