// ipm.cu -- first-order Inverse Polygon Mapping (Sec. 2.3; step 4 of the
// FMM-IPM algorithm of Sec. 2.4).  Each image-plane cell (i, j) of a grid
// chunk has corners y[j][i], y[j][i+1], y[j+1][i+1], y[j+1][i]
// (counter-clockwise in the image plane); its source-plane quadrilateral P
// receives the cell area h^2, apportioned over the map pixels by the signed
// overlap fraction a_pix / A_P, and
//     map[pix] += (h^2 / S*) * a_pix / A_P.
//
// Corners arrive in pixel coordinates u = (y1 - u0)/du, v = (y2 - v0)/dv,
// split as (floor, float fraction) by the deflection epilogue, so no step
// needs float64.  One warp takes 32 consecutive cells
// (k_ipm_cells): single-pixel cells add their whole area; cells with a pixel
// box up to 4 x 4 get one overlap per pixel; larger cells are swept row band
// by row band, whole-pixel runs going to a per-row difference array and
// only the pixels an edge crosses getting an overlap; all three kinds of
// work are spread evenly over the warp's lanes.  Ill-conditioned cells
// (|A_P| small against the box) are queued for float-float (k_ipm_ext).
// Overlaps come from Green's theorem, edge by edge (the apportioning rule of
// Sec. 2.3): the result is the winding-number-weighted area, so inverted and
// self-intersecting (critical) cells are handled "naively", as the
// first-order IPM does.
// Ledger per chunk: area_in_map, area_outside, area_dropped (bbox larger
// than the cap, or a corner beyond 2^30 pixels), area_degenerate
// (|A_P| <= 1e-14 h^2).
#include "cx.cuh"
#include "ipm_warp.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kIpmThreads = 256;
constexpr int kChunksPerGrab = 8;  // 32-cell chunks per fetch of the chunk counter

constexpr int kWarps = kIpmThreads / 32;

// One warp per round of 32 cells of a grid chunk (or of a cell list, or of
// sub-cells given as four corners each), rounds handed out by a counter.
template <bool QUADS, bool LIST = false>
__global__ void __launch_bounds__(kIpmThreads, 4) k_ipm_cells(IpmArgs A) {
  __shared__ WarpCells sh[kWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nchunks = (A.ncells + 31) >> 5;
  const int64_t W = A.nx + 1;
  Ledger led;
  // Chunks of 32 cells are handed out by a counter (qcount[1]), so the
  // warps of a block finish together however the large cells fall; one
  // fetch takes kChunksPerGrab chunks (a single address serves all warps, and
  // a fetch per chunk made it the bound of a pass without B and C work).
  unsigned* next = reinterpret_cast<unsigned*>(A.qcount) + 1;
  unsigned g_u = 0;
  if (lane == 0) g_u = atomicAdd(next, 1u);
  int left = kChunksPerGrab;
  for (int64_t ch = (int64_t)__shfl_sync(0xffffffffu, g_u, 0) * kChunksPerGrab; ch < nchunks;) {
    // the following grab is fetched while this one is processed
    if (lane == 0 && left == kChunksPerGrab) g_u = atomicAdd(next, 1u);
    const int64_t idx = ch * 32 + lane;
    const bool has = idx < A.ncells;
    int64_t c = idx;
    PixCorner q4[4];
    if (has) {
      if (LIST) c = A.cell_list[idx];
      if (QUADS) {
#pragma unroll
        for (int k = 0; k < 4; ++k) q4[k] = A.yc[4 * c + k];
      } else {
        // cell index < 2^30 and nx < 2^31: 32-bit division
        const uint32_t j32 = (uint32_t)c / (uint32_t)A.nx;
        const int64_t j = j32, i = c - j * A.nx;
        q4[0] = A.yc[j * W + i];
        q4[1] = A.yc[j * W + i + 1];
        q4[2] = A.yc[(j + 1) * W + i + 1];
        q4[3] = A.yc[(j + 1) * W + i];
      }
    }
    ipm_round<false>(A, sh[w], lane, has, c, q4, led);
    __syncwarp();  // the next chunk overwrites this one's staging
    if (--left > 0) {
      ++ch;
    } else {
      left = kChunksPerGrab;
      ch = (int64_t)__shfl_sync(0xffffffffu, g_u, 0) * kChunksPerGrab;
    }
  }
  block_add_stats<kWarps>(A.stats, led, A.wcell);
}

// Ill-conditioned cells queued by k_ipm_cells: one warp per cell (ext_cell).
template <bool QUADS>
__global__ void __launch_bounds__(kIpmThreads) k_ipm_ext(IpmArgs A) {
  __shared__ int cut_x[kWarps][64], cut_y[kWarps][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nq = *A.qcount;
  Ledger led;
  for (int64_t t = wg; t < nq; t += nwarps) {
    const int64_t c = A.queue[t];
    PixCorner q4[4];
    if (QUADS) {
#pragma unroll
      for (int k = 0; k < 4; ++k) q4[k] = A.yc[4 * c + k];
    } else {
      const uint32_t j32 = (uint32_t)c / (uint32_t)A.nx;
      const int64_t j = j32, i = c - j * A.nx;
      const int64_t W = A.nx + 1;
      q4[0] = A.yc[j * W + i];
      q4[1] = A.yc[j * W + i + 1];
      q4[2] = A.yc[(j + 1) * W + i + 1];
      q4[3] = A.yc[(j + 1) * W + i];
    }
    ext_cell(A, q4, cut_x[w], cut_y[w], lane, led);
  }
  block_add_stats<kWarps>(A.stats, led, A.wcell);
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

// thresholds and the float32 map increment of a launch (from ip and wcell)
void ipm_prepare(IpmArgs& A) {
  A.thr_area = (float)(1e-13 * A.ip.a_cell / A.ip.s_star);
  A.thr_degen = (float)(1e-14 * A.ip.a_cell / A.ip.s_star);
  A.scale_f = (float)(A.ip.scale * A.wcell);
}

namespace {
void ipm_launch(IpmArgs& A, bool quads, int* qcount, cudaStream_t s,
                std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev) {
  ipm_prepare(A);
  // qcount[0]: float-float queue length; qcount[1]: chunk counter of k_ipm_cells
  LENS_CUDA(cudaMemsetAsync(qcount, 0, 2 * sizeof(int), s));
  std::pair<cudaEvent_t, cudaEvent_t> e;
  if (ev) e = event_pair_begin(s);
  int dev = 0, sms = 152;
  LENS_CUDA(cudaGetDevice(&dev));
  LENS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t chunk_blocks = (A.ncells + kIpmThreads - 1) / kIpmThreads;
  const unsigned g = (unsigned)std::min<int64_t>(chunk_blocks, (int64_t)sms * 8);
  if (quads) k_ipm_cells<true><<<g, kIpmThreads, 0, s>>>(A);
  else if (A.cell_list) k_ipm_cells<false, true><<<g, kIpmThreads, 0, s>>>(A);
  else k_ipm_cells<false><<<g, kIpmThreads, 0, s>>>(A);
  LENS_LAUNCHED("k_ipm_cells");
  if (quads) k_ipm_ext<true><<<sms * 2, kIpmThreads, 0, s>>>(A);
  else k_ipm_ext<false><<<sms * 2, kIpmThreads, 0, s>>>(A);
  LENS_LAUNCHED("k_ipm_ext");
  if (ev) {
    event_pair_end(e, s);
    ev->push_back(e);
  }
}

// Refinement, step 1: for each queued cell, its 3 x 3 corner grid of half
// spacing (the rays to deflect) and the lower-left corners of its 2 x 2
// sub-cells.  A queued cell is a grid cell (origin from the grid) at the first
// level, a sub-cell of the previous level (origin from org_in) after that.
__global__ void k_refine_points(const int* __restrict__ parents, int64_t np,
                                const double2* __restrict__ org_in, double gx0, double gy0,
                                int64_t grow0, int64_t gnx, double h, double2* __restrict__ rays,
                                double2* __restrict__ org_out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int64_t c = parents[k];
  double xl, yl;
  if (org_in) {
    xl = org_in[c].x; yl = org_in[c].y;
  } else {
    // the expression the grid's corners use: x0 + i h, y0 + j h
    const int64_t j = c / gnx, i = c - j * gnx;
    xl = gx0 + (double)i * h; yl = gy0 + (double)(grow0 + j) * h;
  }
  const double g = 0.5 * h;
  const double xs[3] = {xl, xl + g, xl + h}, ys[3] = {yl, yl + g, yl + h};
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) rays[9 * k + 3 * b + a] = make_double2(xs[a], ys[b]);
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 2; ++a) org_out[4 * k + 2 * b + a] = make_double2(xs[a], ys[b]);
}

// Refinement, step 2: the deflected 3 x 3 grids in pixel coordinates, four
// corners (c00, c10, c11, c01) per sub-cell, sub-cell 4k + 2b + a.
__global__ void k_refine_quads(const double2* __restrict__ y, int64_t np, IpmParams ip,
                               PixCorner* __restrict__ quads) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= np * 16) return;
  const int64_t k = t >> 4;
  const int q = (int)(t & 15), sub = q >> 2, corner = q & 3;
  const int a = sub & 1, b = sub >> 1;
  // corner order c00, c10, c11, c01 of the sub-cell at (a, b)
  const int ca = a + (corner == 1 || corner == 2), cb = b + (corner >= 2);
  const double2 p = y[9 * k + 3 * cb + ca];
  const double u = (p.x - ip.u0) * ip.inv_du, v = (p.y - ip.v0) * ip.inv_dv;
  PixCorner pc;
  if (!(fabs(u) < 5.0e8) || !(fabs(v) < 5.0e8)) {
    pc.iu = kFar; pc.fu = 0.f; pc.iv = kFar; pc.fv = 0.f;
  } else {
    const double fu = floor(u), fv = floor(v);
    pc.iu = (int)fu; pc.fu = (float)(u - fu);
    pc.iv = (int)fv; pc.fv = (float)(v - fv);
    // a fraction that rounds up to 1 moves to the next pixel
    if (pc.fu >= 1.f) { pc.iu += 1; pc.fu = 0.f; }
    if (pc.fv >= 1.f) { pc.iv += 1; pc.fv = 0.f; }
  }
  quads[4 * (4 * k + sub) + corner] = pc;
}
}  // namespace

void ipm_accumulate(const PixCorner* yc, int64_t nx, int64_t nrows_cells, const IpmParams& ip,
                    float* map, float* rowdiff, double* stats_dev, int* queue, int* qcount,
                    int* rq, int* rqcount, cudaStream_t s,
                    std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev) {
  const int64_t ncells = nx * nrows_cells;
  if (ncells <= 0) return;
  IpmArgs A{};
  A.yc = yc; A.nx = nx; A.ncells = ncells; A.map = map; A.stats = stats_dev;
  A.D = rowdiff; A.ldd = (int64_t)ip.npx + 1;
  A.queue = queue; A.qcount = qcount; A.ip = ip;
  A.wcell = 1.f;
  A.rq = rq; A.rqcount = rqcount;
  ipm_launch(A, false, qcount, s, ev);
}

void ipm_accumulate_list(const PixCorner* yc, int64_t nx, const int* list, int64_t n,
                         const IpmParams& ip, float* map, float* rowdiff, double* stats_dev,
                         int* queue, int* qcount, int* rq, int* rqcount, cudaStream_t s,
                         std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev) {
  if (n <= 0) return;
  IpmArgs A{};
  A.yc = yc; A.nx = nx; A.ncells = n; A.cell_list = list; A.map = map; A.stats = stats_dev;
  A.D = rowdiff; A.ldd = (int64_t)ip.npx + 1;
  A.queue = queue; A.qcount = qcount; A.ip = ip;
  A.wcell = 1.f;
  A.rq = rq; A.rqcount = rqcount;
  ipm_launch(A, false, qcount, s, ev);
}

int64_t ipm_refine(Plan& P, const int* parents, int64_t np, const double2* org_in, double gx0,
                   double gy0, int64_t grow0, int64_t gnx, double h, int level,
                   const IpmParams& ip, float* map,
                   float* rowdiff, double* stats_dev, int* rq_next, int* rqcount_next,
                   double2* org_out, cudaStream_t s,
                   std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev) {
  if (np <= 0) return 0;
  Scratch rays(&P.da, sizeof(double2) * 9 * (size_t)np);
  Scratch y(&P.da, sizeof(double2) * 9 * (size_t)np);
  Scratch quads(&P.da, sizeof(PixCorner) * 16 * (size_t)np);
  Scratch queue(&P.da, sizeof(int) * 4 * (size_t)np + sizeof(int) * 2);
  k_refine_points<<<grid_for(np, 128), 128, 0, s>>>(parents, np, org_in, gx0, gy0, grow0, gnx,
                                                     h, rays.as<double2>(), org_out);
  LENS_LAUNCHED("k_refine_points");
  evaluate_rays(P, rays.as<double>(), 9 * np, y.as<double>(), nullptr, s);
  k_refine_quads<<<grid_for(16 * np, 256), 256, 0, s>>>(y.as<double2>(), np, ip,
                                                         quads.as<PixCorner>());
  LENS_LAUNCHED("k_refine_quads");
  IpmArgs A{};
  A.yc = quads.as<PixCorner>(); A.nx = 0; A.ncells = 4 * np; A.map = map; A.stats = stats_dev;
  A.D = rowdiff; A.ldd = (int64_t)ip.npx + 1;
  A.queue = queue.as<int>(); A.qcount = queue.as<int>() + 4 * np; A.ip = ip;
  A.wcell = (float)std::ldexp(1.0, -2 * level);
  A.rq = rq_next; A.rqcount = rqcount_next;
  ipm_launch(A, true, A.qcount, s, ev);
  return 4 * np;
}

}  // namespace lens
