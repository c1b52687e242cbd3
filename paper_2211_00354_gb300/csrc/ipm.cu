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
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kIpmThreads = 256;
constexpr int kChunksPerGrab = 8;  // 32-cell chunks per fetch of the chunk counter
constexpr int kFar = 0x7fffffff;

// Twice the mean of clamp(g, 0, 1) for g running linearly from a to b,
// without branches or ordering (the lanes of a warp take different cases):
// 2 (F(b) - F(a)) / (b - a) with F(t) = c^2 / 2 + max(t - 1, 0), c = clamp(t,
// 0, 1), the antiderivative of the clamp.  The difference of squares is
// taken as (c_b - c_a)(c_b + c_a), which keeps its relative precision when
// a and b are close, and max(t - 1, 0) as 2^31 clamp((t - 1) 2^-31, 0, 1),
// exact for t - 1 < 2^31 (pixel-local coordinates are below 2^31): every
// clamp is then a saturating add or fma.  A vanishing b - a (a vertical
// edge) takes twice the clamped midpoint.  All-below-0 gives exactly 0; the
// other pure cases are within an ulp or two.
__device__ __forceinline__ float mean2_clamp01f(float a, float b) {
  constexpr float kS = 4.656612873077393e-10f;  // 2^-31
  const float ca = __saturatef(a), cb = __saturatef(b);
  const float sa = __saturatef(fmaf(a, kS, -kS)), sb = __saturatef(fmaf(b, kS, -kS));
  const float sc = ca + cb;
  const float num = fmaf(cb - ca, sc, (sb - sa) * 4294967296.0f);
  const float d = b - a;
  return fabsf(d) > 1e-30f ? num * frcp_fast(d) : sc;
}

// Signed (winding-weighted) area of the quadrilateral q inside the unit pixel
// [X, X+1] x [Y, Y+1] by Green's theorem: with g(x) = clamp(x - X, 0, 1) on
// the row band Y <= y <= Y+1, dg/dx is the pixel's indicator, so the area is
// the contour integral of g dy; on each straight edge g is piecewise linear,
// giving (y_b - y_a) * mean(g) over the edge's part inside the band.  The
// edge slopes dx/dy are given (0 for a horizontal edge, whose clipped part
// then has ya == yb and adds nothing).
//
// In band-local heights w = y - Y and v = clamp(w, 0, 1) (the clipped
// height), an edge from vertex e to f runs inside the band from v_e to v_f,
// at x - X = (x_e - X) + (v - w_e) dx/dy.
__device__ __forceinline__ float pixel_area_f(const float* qx, const float* qy, const float* sl,
                                              float X, float Y) {
  float w[4], v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w[k] = qy[k] - Y;
    v[k] = __saturatef(w[k]);
  }
  float s = 0.f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int f = (e + 1) & 3;
    const float x0 = qx[e] - X;
    const float ta = fmaf(v[e] - w[e], sl[e], x0), tb = fmaf(v[f] - w[e], sl[e], x0);
    s = fmaf(v[f] - v[e], mean2_clamp01f(ta, tb), s);
  }
  return 0.5f * s;
}

struct IpmArgs {
  const PixCorner* yc;  // (nrows+1) x (nx+1) corners of the chunk, or 4 per cell (quads)
  int64_t nx, ncells;
  float* map;           // float32 accumulation map (added to the float64 output at the end)
  float* D;             // per-row difference array, npy x (npx + 1): prefix-summed at the end
  int64_t ldd;          // npx + 1
  double* stats;        // [8]
  int* queue; int* qcount;   // qcount[0] queue length, qcount[1] chunk counter
  IpmParams ip;
  float thr_area;       // fast-path lower bound on |A_P| in pixel units
  float thr_degen;      // |A_P| (pixel units) at or below which a cell is degenerate
  float scale_f;        // ip.scale x wcell in float32
  float wcell;          // cell area in units of the grid's cell (1, or 4^-level for sub-cells)
  int* rq; int* rqcount;  // refinement: cells over the cap are queued here (NULL: dropped)
};

// Ledger of one thread: fractions in float32, counts in integers (no
// float64 per cell).  Device stats slots: [2] sum of in-map fractions,
// [3] sum of outside fractions (cells wholly outside count 1), [4] dropped
// cells, [5] degenerate cells, [8] map increments, [9] cells on the large-cell
// or float-float path, [10] float-float cells; the host multiplies by the cell area.
struct Ledger {
  float fin = 0.f, fout = 0.f;
  unsigned ndrop = 0, ndeg = 0, nupd = 0, nq = 0, nff = 0;
};

// w: the cells' area in grid cells (uniform over a launch), applied to the
// fractions here once instead of per update.  Slots [6], [7]: dropped and
// degenerate area in grid cells (the counts [4], [5] times w).
__device__ __forceinline__ void block_add_stats(double* stats, const Ledger& L, float wcell) {
  __shared__ float shf[2][kIpmThreads / 32];
  __shared__ unsigned shu[5][kIpmThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float f0 = L.fin, f1 = L.fout;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f0 += __shfl_xor_sync(0xffffffffu, f0, o);
    f1 += __shfl_xor_sync(0xffffffffu, f1, o);
  }
  const unsigned u0 = __reduce_add_sync(0xffffffffu, L.ndrop);
  const unsigned u1 = __reduce_add_sync(0xffffffffu, L.ndeg);
  const unsigned u2 = __reduce_add_sync(0xffffffffu, L.nupd);
  const unsigned u3 = __reduce_add_sync(0xffffffffu, L.nq);
  const unsigned u4 = __reduce_add_sync(0xffffffffu, L.nff);
  if (lane == 0) {
    shf[0][w] = f0; shf[1][w] = f1;
    shu[0][w] = u0; shu[1][w] = u1; shu[2][w] = u2; shu[3][w] = u3; shu[4][w] = u4;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    // thread t: slots 2, 3 (fractions x w), 4, 5 (counts), 8, 9, 10, then 6, 7
    const int src = threadIdx.x < 7 ? threadIdx.x : threadIdx.x - 5;
    double x = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
      x += src < 2 ? (double)shf[src][q] : (double)shu[src - 2][q];
    if (src < 2 || threadIdx.x >= 7) x *= (double)wcell;
    const int slot = threadIdx.x < 4 ? 2 + threadIdx.x : threadIdx.x < 7 ? 4 + threadIdx.x : threadIdx.x - 1;
    if (x != 0.0) atomicAdd(&stats[slot], x);
  }
}

// Does the segment P->Q meet the closed unit square at (ox, oy)?  (float32
// pre-filter for the float-float path: a pixel that no edge meets is covered by
// the polygon's winding number exactly.)
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
  // a margin covers float32 rounding of the corners: near-misses count as hits
  const float tol = 1e-5f * (fabsf(dx) + fabsf(dy)) * (1.f + fabsf(ox) + fabsf(oy));
  return !(lo > tol || hi < -tol);
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

// Inclusive warp scan of per-lane counts; cum[] receives the 32 inclusive
// sums, the return value is the warp total.
__device__ __forceinline__ int warp_counts(int cnt, int* cum, int lane) {
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  cum[lane] = incl;
  __syncwarp();
  return __shfl_sync(0xffffffffu, incl, 31);
}
// Owner of flat task f: the first lane whose inclusive count exceeds f, and
// f's offset within that lane's tasks.
__device__ __forceinline__ int warp_owner(const int* cum, int f, int& off) {
  int L = 0;
#pragma unroll
  for (int st = 16; st > 0; st >>= 1)
    if (cum[L + st - 1] <= f) L += st;
  off = f - (L ? cum[L - 1] : 0);
  return L;
}

constexpr int kSmallBox = 4;  // pixel boxes up to 4 x 4: overlap pixel by pixel
constexpr int kWarps = kIpmThreads / 32;

// Per-warp staging: the warp's 32 cells, then up to 32 rows x 4 edge
// segments of large cells.
struct CellShared {
  float4 qx[kWarps][32], qy[kWarps][32];  // polygon, pixel units local to (ix0, iy0)
  float4 sl[kWarps][32];                  // edge slopes dx/dy (0 if horizontal)
  int4 box[kWarps][32];                   // ix0, iy0, cx0, cy0 (box clipped to the map at cx0, cy0)
  int2 ext[kWarps][32];                   // clipped box width (+ whole-box flag and height
                                          // of a small cell), 1 / A_P (float bits)
  int cum[kWarps][32], cum2[kWarps][32];
  // owner lane of each (cell, pixel) task of the small cells (<= 32 x 16)
  unsigned char own[kWarps][32 * kSmallBox * kSmallBox];
  float4 seg[kWarps][128];                // crossing segments: xa, xb, dy / 2, first pixel (int bits)
  int4 sst[kWarps][32];                   // starts of a row task's segments 1..3 in its pixel list
  int2 rbi[kWarps][32];                   // row task: map offset of (row, box x0), 1 / A_P (float bits)
};

__device__ __forceinline__ void unpack4(float (&a)[4], const float4 v) {
  a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
}

// One warp per 32 consecutive cells of a grid row (grid-stride over chunks).
//  A. lane = cell: corners (coalesced), pixel box, ledger of cells that are
//     dropped or outside, single-pixel cells (fraction 1), hand-off of
//     ill-conditioned cells to the float-float queue;
//  B. small cells (box <= 4 x 4): the warp's (cell, pixel) pairs spread over
//     the lanes, one Green's-theorem overlap each (a box inside the map skips
//     its last pixel, which takes the remainder of the cell);
//  C. large cells: the warp's (cell, row) pairs spread over the lanes; in the
//     band Y <= y <= Y+1 an edge whose clipped part runs (xa,ya)->(xb,yb)
//     adds dy = yb - ya to each pixel X with X + 1 <= min(xa, xb): that
//     whole-pixel run enters the per-row difference array as +v / -v at its
//     ends, and only the pixels the segment crosses get an explicit overlap
//     (the same Green's-theorem terms as pixel_area_f()), again spread over
//     the lanes.  Work per large cell follows its perimeter in pixels, not
//     its area.
template <bool QUADS>
__global__ void __launch_bounds__(kIpmThreads, 4) k_ipm_cells(IpmArgs A) {
  __shared__ CellShared sh;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nchunks = (A.ncells + 31) >> 5;
  const int64_t W = A.nx + 1;
  const int npx = A.ip.npx, npy = A.ip.npy;
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
    // ---- A: one cell per lane ------------------------------------------------
    const int64_t c = ch * 32 + lane;
    int nsmall = 0, nrows = 0;
    bool f64 = false;
    if (c < A.ncells) {
      PixCorner q4[4];
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
      bool far = false;
      int ix0 = kFar, ix1 = -kFar, iy0 = kFar, iy1 = -kFar;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        far |= (q4[k].iu == kFar) | (q4[k].iv == kFar);
        ix0 = min(ix0, q4[k].iu); ix1 = max(ix1, q4[k].iu);
        iy0 = min(iy0, q4[k].iv); iy1 = max(iy1, q4[k].iv);
      }
      if (!far && (ix1 < 0 || iy1 < 0 || ix0 > npx - 1 || iy0 > npy - 1)) {
        led.fout += 1.f;
      } else if (far || (A.ip.cap > 0 && ((int64_t)ix1 - ix0 + 1 > A.ip.cap ||
                                          (int64_t)iy1 - iy0 + 1 > A.ip.cap))) {
        // over the cap (or a corner beyond 2^30 pixels): split further, or dropped
        if (A.rq) A.rq[atomicAdd(A.rqcount, 1)] = (int)c;
        else led.ndrop += 1;
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
        const bool good = fabsf(A_loc) > 1e-3f * (xmx - xmn) * (ymx - ymn) && fabsf(A_loc) > A.thr_area;
        if (!good) {
          f64 = true;
          led.nq += 1;
        } else if (ix0 == ix1 && iy0 == iy1) {
          atomicAdd(&A.map[(int64_t)iy0 * npx + ix0], A.scale_f);
          led.fin += 1.f;
          led.nupd += 1;
        } else {
          const int cx0 = max(ix0, 0), cx1 = min(ix1, npx - 1);
          const int cy0 = max(iy0, 0), cy1 = min(iy1, npy - 1);
          float slk[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            // an edge with |dy| <= 1e-30 adds nothing (its clipped dy is at
            // most that): slope 0 keeps its terms finite
            const float ey = qy[(k + 1) & 3] - qy[k];
            slk[k] = fabsf(ey) > 1e-30f ? __fdividef(qx[(k + 1) & 3] - qx[k], ey) : 0.f;
          }
          sh.qx[w][lane] = make_float4(qx[0], qx[1], qx[2], qx[3]);
          sh.qy[w][lane] = make_float4(qy[0], qy[1], qy[2], qy[3]);
          sh.sl[w][lane] = make_float4(slk[0], slk[1], slk[2], slk[3]);
          sh.box[w][lane] = make_int4(ix0, iy0, cx0, cy0);
          const bool smallc = ix1 - ix0 < kSmallBox && iy1 - iy0 < kSmallBox;
          // A small cell whose pixel box lies inside the map puts all of its
          // area there: its fractions sum to 1 (winding-weighted areas add up
          // to the signed area), so the last pixel of the box is not
          // evaluated and takes 1 minus the others (added whole here, each
          // other pixel's fraction subtracted from it in B).
          const bool whole = smallc && cx0 == ix0 && cy0 == iy0 && cx1 == ix1 && cy1 == iy1;
          // |A_loc| > 0: the cell is well conditioned
          sh.ext[w][lane] = make_int2((cx1 - cx0 + 1) | (whole ? (cy1 - cy0 + 1) << 3 : 0),
                                      __float_as_int(frcp_fast(A_loc)));
          if (whole) {
            atomicAdd(&A.map[(int64_t)cy1 * npx + cx1], A.scale_f);
            led.fin += 1.f;
            led.nupd += 1;
          } else {
            // every fraction that lands in the map is moved from fout to fin
            led.fout += 1.f;
          }
          if (smallc) {
            nsmall = (cx1 - cx0 + 1) * (cy1 - cy0 + 1) - (whole ? 1 : 0);
          } else {
            nrows = cy1 - cy0 + 1;
            led.nq += 1;
          }
        }
      }
    }
    // ill-conditioned cells: one queue slot per cell, one atomic per warp
    const unsigned fm = __ballot_sync(0xffffffffu, f64);
    if (fm) {
      int base = 0;
      if (lane == 0) base = atomicAdd(A.qcount, __popc(fm));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (f64) A.queue[base + __popc(fm & ((1u << lane) - 1u))] = (int)c;
    }
    // ---- B: pixels of small cells -------------------------------------------
    const int tot1 = warp_counts(nsmall, sh.cum[w], lane);
    {
      // each lane marks its tasks with its index: one byte load finds a
      // task's cell
      const int st = sh.cum[w][lane] - nsmall;
      for (int i = 0; i < nsmall; ++i) sh.own[w][st + i] = (unsigned char)lane;
      __syncwarp();
    }
    for (int f0 = 0; f0 < tot1; f0 += 32) {
      const int f = f0 + lane;
      if (f < tot1) {
        const int L = sh.own[w][f];
        const int off = f - (L ? sh.cum[w][L - 1] : 0);
        const int4 bx = sh.box[w][L];
        const int2 ex = sh.ext[w][L];
        const int wd = ex.x & 7, hg = ex.x >> 3;  // hg > 0: a whole-box cell of hg rows
        // off < 16 and wd <= 4: off / wd without a division
        const int r = wd == 3 ? (off * 21846) >> 16 : off >> (wd >> 1);
        const int px = bx.z + off - r * wd, py = bx.w + r;
        float qx[4], qy[4], sl[4];
        unpack4(qx, sh.qx[w][L]);
        unpack4(qy, sh.qy[w][L]);
        unpack4(sl, sh.sl[w][L]);
        const float a = pixel_area_f(qx, qy, sl, (float)(px - bx.x), (float)(py - bx.y));
        if (a != 0.0f) {
          const float fr = a * __int_as_float(ex.y);
          atomicAdd(&A.map[(int64_t)py * npx + px], A.scale_f * fr);
          led.nupd += 1;
          if (hg) {
            // inside the map: npx * npy < 2^31, the offset fits an int (the
            // remainder's correction, not counted as a map increment)
            atomicAdd(&A.map[(bx.w + hg - 1) * npx + bx.z + wd - 1], -A.scale_f * fr);
          } else {
            led.fin += fr;
            led.fout -= fr;
          }
        }
      }
    }
    // ---- C: rows of large cells ---------------------------------------------
    const int tot2 = warp_counts(nrows, sh.cum2[w], lane);
    for (int f0 = 0; f0 < tot2; f0 += 32) {
      const int f = f0 + lane;
      int cnt = 0;
      if (f < tot2) {
        int r;
        const int L = warp_owner(sh.cum2[w], f, r);
        const int4 bx = sh.box[w][L];
        const int2 ex = sh.ext[w][L];
        const int ix0 = bx.x, cx0 = bx.z;
        const int lx0 = cx0 - ix0, lx1 = lx0 + ex.x - 1;
        const float inv = __int_as_float(ex.y);
        const float kf = A.scale_f * inv;  // map increment per unit of pixel area
        const int py = bx.w + r;
        const float Y = (float)(py - bx.y);
        const int64_t drow = (int64_t)py * A.ldd;
        float qx[4], qy[4], slp[4];
        unpack4(qx, sh.qx[w][L]);
        unpack4(qy, sh.qy[w][L]);
        unpack4(slp, sh.sl[w][L]);
        float vsum = 0.f, frow = 0.f;
        int st[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int t = lane * 4 + e;
          int n = 0;
          st[e] = cnt;
          const float x0 = qx[e], y0 = qy[e];
          const float y1 = qy[(e + 1) & 3];
          const float ya = fminf(fmaxf(y0, Y), Y + 1.f), yb = fminf(fmaxf(y1, Y), Y + 1.f);
          if (ya != yb) {
            // the clipped segment of pixel_area_f()
            const float sl = slp[e];
            const float xa = x0 + (ya - y0) * sl, xb = x0 + (yb - y0) * sl;
            const float dy = yb - ya;
            const int Xa = (int)floorf(fminf(xa, xb)), Xb = (int)ceilf(fmaxf(xa, xb)) - 1;
            // whole-pixel run [lx0, Xa): each pixel gains dy
            const int hi = min(Xa, lx1 + 1);
            if (hi > lx0) {
              const float v = dy * kf;
              atomicAdd(&A.D[drow + ix0 + hi], -v);
              vsum += v;
              frow += dy * (float)(hi - lx0);
              led.nupd += 1;
            }
            // pixels the segment crosses: [max(Xa, lx0), min(Xb, lx1)]
            const int pa = max(Xa, lx0), pb = min(Xb, lx1);
            if (pb >= pa) {
              n = pb - pa + 1;
              sh.seg[w][t] = make_float4(xa, xb, 0.5f * dy, __int_as_float(pa));
            }
          }
          cnt += n;
        }
        if (vsum != 0.f) { atomicAdd(&A.D[drow + cx0], vsum); led.nupd += 1; }
        led.fin += frow * inv;
        led.fout -= frow * inv;
        sh.sst[w][lane] = make_int4(st[1], st[2], st[3], cnt);
        // npx * npy < 2^31 and |ix0| < 2^30: the offset fits an int
        sh.rbi[w][lane] = make_int2(py * npx + ix0, __float_as_int(inv));
      }
      // crossed pixels of these 32 rows, spread over the lanes
      int* cum = sh.cum[w];  // the small-cell counts are no longer needed
      __syncwarp();
      const int totp = warp_counts(cnt, cum, lane);
      for (int g0 = 0; g0 < totp; g0 += 32) {
        const int g = g0 + lane;
        if (g < totp) {
          int off;
          const int L = warp_owner(cum, g, off);
          // segment k of row task L: the last one starting at or before off
          // (an empty segment shares its start with the next one)
          const int4 ss = sh.sst[w][L];
          const int k = (off >= ss.x) + (off >= ss.y) + (off >= ss.z);
          off -= k == 0 ? 0 : k == 1 ? ss.x : k == 2 ? ss.y : ss.z;
          const float4 sg = sh.seg[w][L * 4 + k];
          const int X = __float_as_int(sg.w) + off;
          const float a = sg.z * mean2_clamp01f(sg.x - (float)X, sg.y - (float)X);
          if (a != 0.0f) {
            const int2 rb = sh.rbi[w][L];
            const float fr = a * __int_as_float(rb.y);
            atomicAdd(&A.map[rb.x + X], A.scale_f * fr);
            led.fin += fr;
            led.fout -= fr;
            led.nupd += 1;
          }
        }
      }
      __syncwarp();
    }
    __syncwarp();  // the next chunk overwrites this one's staging
    if (--left > 0) {
      ++ch;
    } else {
      left = kChunksPerGrab;
      ch = (int64_t)__shfl_sync(0xffffffffu, g_u, 0) * kChunksPerGrab;
    }
  }
  block_add_stats(A.stats, led, A.wcell);
}

// ---- float-float (about 48-bit) arithmetic for ill-conditioned cells -------
// The pieces of lens::ff (cx.cuh) plus subtraction, order and division, all
// on the float32 pipe (the float64 pipe is ~60x slower on this GPU).
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.hi, -b.lo}); }
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ ff ff_min(ff a, ff b) { return ff_lt(b, a) ? b : a; }
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }
__device__ __forceinline__ ff ff_div(ff a, ff b) {  // b != 0
  const float q1 = a.hi / b.hi;
  const ff r = ff_sub(a, ff_mul(b, q1));
  return ff_norm(q1, r.hi / b.hi);
}
__device__ __forceinline__ ff ff_half(ff a) { return ff{0.5f * a.hi, 0.5f * a.lo}; }

// mean_clamp01f() in float-float.
__device__ __forceinline__ ff mean_clamp01_ff(ff a, ff b) {
  const ff zero{0.f, 0.f}, one{1.f, 0.f};
  const ff lo = ff_min(a, b), hi = ff_max(a, b);
  const ff l0 = ff_max(lo, zero), h1 = ff_min(hi, one);
  const ff I = ff_add(ff_mul(ff_half(ff_max(ff_sub(h1, l0), zero)), ff_add(h1, l0)),
                      ff_max(ff_sub(hi, ff_max(lo, one)), zero));
  const ff d = ff_sub(hi, lo);
  if (d.hi > 1e-30f) return ff_div(I, d);
  return ff_min(ff_max(ff_half(ff_add(lo, hi)), zero), one);
}

// pixel_area_f() in float-float, slopes given (0 for a horizontal edge)
__device__ __forceinline__ ff pixel_area_ff(const ff* qx, const ff* qy, const ff* sl, int X, int Y) {
  const ff Yl{(float)Y, 0.f}, Yh{(float)(Y + 1), 0.f};
  ff s{0.f, 0.f};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const ff y0 = qy[e], y1 = qy[(e + 1) & 3];
    const ff ya = ff_min(ff_max(y0, Yl), Yh), yb = ff_min(ff_max(y1, Yl), Yh);
    if (ya.hi == yb.hi && ya.lo == yb.lo) continue;
    const ff xa = ff_add(qx[e], ff_mul(ff_sub(ya, y0), sl[e]));
    const ff xb = ff_add(qx[e], ff_mul(ff_sub(yb, y0), sl[e]));
    const ff m = mean_clamp01_ff(ff_add(xa, -(float)X), ff_add(xb, -(float)X));
    s = ff_add(s, ff_mul(ff_sub(yb, ya), m));
  }
  return s;
}

// Ill-conditioned cells (|A_P| small against the pixel box): one warp per
// cell, lanes over the box's pixels.  A float32 test finds the pixels no
// edge meets, whose coverage is the winding number exactly; the pixels an
// edge cuts are collected in shared memory and their overlaps taken in
// float-float (coordinates local to the box, exact from the corners' integer
// and fractional parts) 32 at a time.
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
    int ix0 = kFar, ix1 = -kFar, iy0 = kFar, iy1 = -kFar;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ix0 = min(ix0, q4[k].iu); ix1 = max(ix1, q4[k].iu);
      iy0 = min(iy0, q4[k].iv); iy1 = max(iy1, q4[k].iv);
    }
    const int cx0 = max(ix0, 0), cx1 = min(ix1, A.ip.npx - 1);
    const int cy0 = max(iy0, 0), cy1 = min(iy1, A.ip.npy - 1);
    const int wd = cx1 - cx0 + 1;
    const int npix = wd * (cy1 - cy0 + 1);  // the box is at most cap x cap, or clipped to the map
    float fx[4], fy[4];
    ff u[4], v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      fx[k] = (float)(q4[k].iu - ix0) + q4[k].fu;
      fy[k] = (float)(q4[k].iv - iy0) + q4[k].fv;
      // integer part (< 2^24 in the box) + fraction: exact as a two-sum
      float sh, eh;
      two_sum((float)(q4[k].iu - ix0), q4[k].fu, sh, eh);
      u[k] = ff{sh, eh};
      two_sum((float)(q4[k].iv - iy0), q4[k].fv, sh, eh);
      v[k] = ff{sh, eh};
    }
    // shoelace over the diagonals: 2 A_P = (u2-u0)(v3-v1) - (u3-u1)(v2-v0)
    const ff A_P = ff_half(ff_sub(ff_mul(ff_sub(u[2], u[0]), ff_sub(v[3], v[1])),
                                  ff_mul(ff_sub(u[3], u[1]), ff_sub(v[2], v[0]))));
    if (!(fabsf(A_P.hi) > A.thr_degen)) {
      if (lane == 0) led.ndeg += 1;
      continue;
    }
    if (lane == 0) led.nff += 1;
    const ff inv = ff_div(ff{1.f, 0.f}, A_P);
    ff sl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const ff ey = ff_sub(v[(k + 1) & 3], v[k]);
      sl[k] = ey.hi != 0.f ? ff_div(ff_sub(u[(k + 1) & 3], u[k]), ey) : ff{0.f, 0.f};
    }
    const float invf = inv.hi;
    float fin = 0.f;
    int ncut = 0;  // warp-uniform: entries waiting in cut_x[w], cut_y[w]
    for (int base = 0; base < npix; base += 32) {
      const int t2 = base + lane;
      bool cut = false;
      int ox = 0, oy = 0;
      if (t2 < npix) {
        const int r = t2 / wd;
        oy = cy0 - iy0 + r;
        ox = cx0 - ix0 + (t2 - r * wd);
#pragma unroll
        for (int e = 0; e < 4; ++e)
          cut |= seg_meets_pixel(fx[e], fy[e], fx[(e + 1) & 3], fy[(e + 1) & 3], (float)ox, (float)oy);
        if (!cut) {
          const int wn = winding4(fx, fy, (float)ox + 0.5f, (float)oy + 0.5f);
          const float fr = (float)wn * invf;
          if (fr != 0.0f) {
            atomicAdd(&A.map[(int64_t)(iy0 + oy) * A.ip.npx + ix0 + ox], A.scale_f * fr);
            fin += fr;
            led.nupd += 1;
          }
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, cut);
      if (cut) {
        const int slot = ncut + __popc(m & ((1u << lane) - 1u));  // < 64: ncut < 32 here
        cut_x[w][slot] = ox;
        cut_y[w][slot] = oy;
      }
      ncut += __popc(m);
      const bool last = base + 32 >= npix;
      while (ncut >= 32 || (last && ncut > 0)) {
        __syncwarp();
        const int take = min(ncut, 32);
        if (lane < take) {
          const int px = cut_x[w][lane], py = cut_y[w][lane];
          const float fr = ff_mul(pixel_area_ff(u, v, sl, px, py), inv).hi;
          if (fr != 0.0f) {
            atomicAdd(&A.map[(int64_t)(iy0 + py) * A.ip.npx + ix0 + px], A.scale_f * fr);
            fin += fr;
            led.nupd += 1;
          }
        }
        __syncwarp();
        // move the rest (at most 31) to the front
        const int rest = ncut - take;
        int kx = 0, ky = 0;
        if (lane < rest) { kx = cut_x[w][take + lane]; ky = cut_y[w][take + lane]; }
        __syncwarp();
        if (lane < rest) { cut_x[w][lane] = kx; cut_y[w][lane] = ky; }
        __syncwarp();
        ncut = rest;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fin += __shfl_xor_sync(0xffffffffu, fin, o);
    if (lane == 0) { led.fin += fin; led.fout += 1.f - fin; }
  }
  block_add_stats(A.stats, led, A.wcell);
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

// map (+)= map32 + row-wise prefix sum of the difference array (float64),
// one block per map row: each thread sums a contiguous run of columns, a
// block scan gives each run its offset, and the run is written out.  With
// `clear` the float32 accumulators are zeroed behind the read, so the next
// cells start from zero (a flush between chunks).
constexpr int kFinishThreads = 256;

__global__ void __launch_bounds__(kFinishThreads)
k_map_finish(float* __restrict__ m32, float* __restrict__ D, int npx, int npy, int64_t ldd,
             double* __restrict__ out, bool accumulate, bool clear) {
  __shared__ double wsum[kFinishThreads / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int run = (npx + kFinishThreads - 1) / kFinishThreads;
  const int c0 = min(npx, t * run), c1 = min(npx, c0 + run);
  for (int64_t row = blockIdx.x; row < npy; row += gridDim.x) {
    float* d = D + row * ldd;
    double s = 0.0;
    for (int c = c0; c < c1; ++c) s += (double)d[c];
    double incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    __syncthreads();  // the previous row's readers of wsum are done
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    double base = incl - s;
    for (int q = 0; q < w; ++q) base += wsum[q];
    float* m = m32 + row * (int64_t)npx;
    double* o = out + row * (int64_t)npx;
    for (int c = c0; c < c1; ++c) {
      base += (double)d[c];
      const double v = (double)m[c] + base;
      o[c] = accumulate ? o[c] + v : v;
      if (clear) { m[c] = 0.f; d[c] = 0.f; }
    }
    // column npx of the difference array only ever receives run ends
    if (clear && t == 0) d[npx] = 0.f;
  }
}

void ipm_finish_map(float* map32, float* rowdiff, int npx, int npy, double* map, bool accumulate,
                    bool clear, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<int64_t>(npy, 152 * 8);
  k_map_finish<<<blocks, kFinishThreads, 0, s>>>(map32, rowdiff, npx, npy, (int64_t)npx + 1, map,
                                                 accumulate, clear);
  LENS_LAUNCHED("k_map_finish");
}

namespace {
void ipm_launch(IpmArgs& A, bool quads, int* qcount, cudaStream_t s,
                std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev) {
  A.thr_area = (float)(1e-13 * A.ip.a_cell / A.ip.s_star);
  A.thr_degen = (float)(1e-14 * A.ip.a_cell / A.ip.s_star);
  A.scale_f = (float)(A.ip.scale * A.wcell);
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
