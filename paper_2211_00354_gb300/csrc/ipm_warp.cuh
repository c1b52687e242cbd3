// ipm_warp.cuh -- the warp-level core of the first-order IPM (Sec. 2.3, the
// apportioning of a mapped cell's area over the map pixels by Green's
// theorem; step 4 of the FMM-IPM algorithm of Sec. 2.4), shared by the IPM
// kernels (ipm.cu) and the fused deflection + IPM kernel (fused.cu).
//
// ipm_round() maps one round of 32 cells, one per lane, whose corners the
// caller has loaded in pixel coordinates: single-pixel cells add their whole
// weight; cells whose pixel box is at most 4 x 4 get one Green's-theorem
// overlap per pixel, the (cell, pixel) pairs spread over the lanes; larger
// cells are swept row band by row band, whole-pixel runs entering a per-row
// difference array and only the pixels an edge crosses getting an overlap,
// again spread over the lanes; ill-conditioned cells are queued for the
// float-float path.  Every map update is a float32 atomic add.
#pragma once

#include "cx.cuh"
#include "lens_internal.h"

namespace lens {

constexpr int kFar = 0x7fffffff;
constexpr int kSmallBox = 4;  // pixel boxes up to 4 x 4: overlap pixel by pixel

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
  const int* cell_list;   // k_ipm_cells: the cells to map (ids into yc's grid), or NULL: all
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

// Per-warp staging of a round: its 32 cells, then up to 32 rows x 4 edge
// segments of large cells.
struct WarpCells {
  float4 qx[32], qy[32];  // polygon, pixel units local to (ix0, iy0)
  float4 sl[32];          // edge slopes dx/dy (0 if horizontal)
  int4 box[32];           // ix0, iy0, cx0, cy0 (box clipped to the map at cx0, cy0)
  int2 ext[32];           // clipped box width (+ whole-box flag and height
                          // of a small cell), 1 / A_P (float bits)
  int cum[32], cum2[32];
  // owner lane of each (cell, pixel) task of the small cells (<= 32 x 16)
  unsigned char own[32 * kSmallBox * kSmallBox];
  float4 seg[128];        // crossing segments: xa, xb, dy / 2, first pixel (int bits)
  int4 sst[32];           // starts of a row task's segments 1..3 in its pixel list
  int2 rbi[32];           // row task: map offset of (row, box x0), 1 / A_P (float bits)
};

namespace {

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





// w: the cells' area in grid cells (uniform over a launch), applied to the
// fractions here once instead of per update.  Slots [6], [7]: dropped and
// degenerate area in grid cells (the counts [4], [5] times w).
template <int NW>
__device__ __forceinline__ void block_add_stats(double* stats, const Ledger& L, float wcell) {
  __shared__ float shf[2][NW];
  __shared__ unsigned shu[5][NW];
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
    for (int q = 0; q < NW; ++q)
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



__device__ __forceinline__ void unpack4(float (&a)[4], const float4 v) {
  a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
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

// One ill-conditioned cell (|A_P| small against its pixel box) by the whole
// warp, lanes over the box's pixels: a float32 test finds the pixels no edge
// meets, whose coverage is the winding number exactly; the pixels an edge
// cuts are collected in cut_x / cut_y (the warp's 64 slots) and their
// overlaps taken in float-float (coordinates local to the box, exact from the
// corners' integer and fractional parts) 32 at a time.  q4: the cell's
// corners (the same in every lane).
template <bool INLINE>
__device__ __forceinline__ void ext_cell_body(const IpmArgs& A, const PixCorner (&q4)[4], int* cut_x,
                                              int* cut_y, int lane, Ledger& led) {
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
    return;
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
  int ncut = 0;  // warp-uniform: entries waiting in cut_x, cut_y
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
      cut_x[slot] = ox;
      cut_y[slot] = oy;
    }
    ncut += __popc(m);
    const bool last = base + 32 >= npix;
    while (ncut >= 32 || (last && ncut > 0)) {
      __syncwarp();
      const int take = min(ncut, 32);
      if (lane < take) {
        const int px = cut_x[lane], py = cut_y[lane];
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
      if (lane < rest) { kx = cut_x[take + lane]; ky = cut_y[take + lane]; }
      __syncwarp();
      if (lane < rest) { cut_x[lane] = kx; cut_y[lane] = ky; }
      __syncwarp();
      ncut = rest;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fin += __shfl_xor_sync(0xffffffffu, fin, o);
  if (lane == 0) { led.fin += fin; led.fout += 1.f - fin; }
}

__device__ __forceinline__ void ext_cell(const IpmArgs& A, const PixCorner (&q4)[4], int* cut_x,
                                         int* cut_y, int lane, Ledger& led) {
  ext_cell_body<true>(A, q4, cut_x, cut_y, lane, led);
}
// the same as a call (rare cells; keeps its registers out of the caller's)
__device__ __noinline__ void ext_cell_call(const IpmArgs& A, const PixCorner* q4, int* cut_x,
                                           int* cut_y, int lane, Ledger& led) {
  const PixCorner q[4] = {q4[0], q4[1], q4[2], q4[3]};
  ext_cell_body<false>(A, q, cut_x, cut_y, lane, led);
}

// One round of 32 cells (lane = cell; `has`: the lane holds a cell, `c` its
// id for the queues, q4 its corners c00, c10, c11, c01 in pixel coordinates):
//  A. lane = cell: pixel box, ledger of cells that are dropped or outside,
//     single-pixel cells (fraction 1), hand-off of ill-conditioned cells to
//     the float-float path (queued by id for k_ipm_ext, or with EXT mapped
//     by the whole warp before the round goes on);
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
template <bool EXT>
__device__ __forceinline__ void ipm_round(const IpmArgs& A, WarpCells& sh, int lane, bool has,
                                          int64_t c, const PixCorner (&q4)[4], Ledger& led,
                                          int* cut = nullptr) {
  const int npx = A.ip.npx, npy = A.ip.npy;
  // ---- A: one cell per lane ------------------------------------------------
  int nsmall = 0, nrows = 0;
  bool f64 = false;
  if (has) {
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
        sh.qx[lane] = make_float4(qx[0], qx[1], qx[2], qx[3]);
        sh.qy[lane] = make_float4(qy[0], qy[1], qy[2], qy[3]);
        sh.sl[lane] = make_float4(slk[0], slk[1], slk[2], slk[3]);
        sh.box[lane] = make_int4(ix0, iy0, cx0, cy0);
        const bool smallc = ix1 - ix0 < kSmallBox && iy1 - iy0 < kSmallBox;
        // A small cell whose pixel box lies inside the map puts all of its
        // area there: its fractions sum to 1 (winding-weighted areas add up
        // to the signed area), so the last pixel of the box is not
        // evaluated and takes 1 minus the others (added whole here, each
        // other pixel's fraction subtracted from it in B).
        const bool whole = smallc && cx0 == ix0 && cy0 == iy0 && cx1 == ix1 && cy1 == iy1;
        // |A_loc| > 0: the cell is well conditioned
        sh.ext[lane] = make_int2((cx1 - cx0 + 1) | (whole ? (cy1 - cy0 + 1) << 3 : 0),
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
  // ill-conditioned cells: queued for the float-float kernel (one queue slot
  // per cell, one atomic per warp), or with EXT mapped here by the whole
  // warp, one cell after another
  const unsigned fm = __ballot_sync(0xffffffffu, f64);
  if (EXT) {
    for (unsigned m = fm; m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      PixCorner qq[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        qq[k].iu = __shfl_sync(0xffffffffu, q4[k].iu, src);
        qq[k].fu = __shfl_sync(0xffffffffu, q4[k].fu, src);
        qq[k].iv = __shfl_sync(0xffffffffu, q4[k].iv, src);
        qq[k].fv = __shfl_sync(0xffffffffu, q4[k].fv, src);
      }
      ext_cell_call(A, qq, cut, cut + 64, lane, led);
    }
  } else if (fm) {
    int base = 0;
    if (lane == 0) base = atomicAdd(A.qcount, __popc(fm));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (f64) A.queue[base + __popc(fm & ((1u << lane) - 1u))] = (int)c;
  }
  // ---- B: pixels of small cells (skipped by a round without any) ----------
  if (__any_sync(0xffffffffu, nsmall > 0)) {
    const int tot1 = warp_counts(nsmall, sh.cum, lane);
    {
      // each lane marks its tasks with its index: one byte load finds a
      // task's cell
      const int st = sh.cum[lane] - nsmall;
      for (int i = 0; i < nsmall; ++i) sh.own[st + i] = (unsigned char)lane;
      __syncwarp();
    }
    for (int f0 = 0; f0 < tot1; f0 += 32) {
      const int f = f0 + lane;
      if (f < tot1) {
        const int L = sh.own[f];
        const int off = f - (L ? sh.cum[L - 1] : 0);
        const int4 bx = sh.box[L];
        const int2 ex = sh.ext[L];
        const int wd = ex.x & 7, hg = ex.x >> 3;  // hg > 0: a whole-box cell of hg rows
        // off < 16 and wd <= 4: off / wd without a division
        const int r = wd == 3 ? (off * 21846) >> 16 : off >> (wd >> 1);
        const int px = bx.z + off - r * wd, py = bx.w + r;
        float qx[4], qy[4], sl[4];
        unpack4(qx, sh.qx[L]);
        unpack4(qy, sh.qy[L]);
        unpack4(sl, sh.sl[L]);
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
  }
  // ---- C: rows of large cells (skipped by a round without any) -------------
  if (!__any_sync(0xffffffffu, nrows > 0)) return;
  const int tot2 = warp_counts(nrows, sh.cum2, lane);
  for (int f0 = 0; f0 < tot2; f0 += 32) {
    const int f = f0 + lane;
    int cnt = 0;
    if (f < tot2) {
      int r;
      const int L = warp_owner(sh.cum2, f, r);
      const int4 bx = sh.box[L];
      const int2 ex = sh.ext[L];
      const int ix0 = bx.x, cx0 = bx.z;
      const int lx0 = cx0 - ix0, lx1 = lx0 + ex.x - 1;
      const float inv = __int_as_float(ex.y);
      const float kf = A.scale_f * inv;  // map increment per unit of pixel area
      const int py = bx.w + r;
      const float Y = (float)(py - bx.y);
      const int64_t drow = (int64_t)py * A.ldd;
      float qx[4], qy[4], slp[4];
      unpack4(qx, sh.qx[L]);
      unpack4(qy, sh.qy[L]);
      unpack4(slp, sh.sl[L]);
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
            sh.seg[t] = make_float4(xa, xb, 0.5f * dy, __int_as_float(pa));
          }
        }
        cnt += n;
      }
      if (vsum != 0.f) { atomicAdd(&A.D[drow + cx0], vsum); led.nupd += 1; }
      led.fin += frow * inv;
      led.fout -= frow * inv;
      sh.sst[lane] = make_int4(st[1], st[2], st[3], cnt);
      // npx * npy < 2^31 and |ix0| < 2^30: the offset fits an int
      sh.rbi[lane] = make_int2(py * npx + ix0, __float_as_int(inv));
    }
    // crossed pixels of these 32 rows, spread over the lanes
    int* cum = sh.cum;  // the small-cell counts are no longer needed
    __syncwarp();
    const int totp = warp_counts(cnt, cum, lane);
    for (int g0 = 0; g0 < totp; g0 += 32) {
      const int g = g0 + lane;
      if (g < totp) {
        int off;
        const int L = warp_owner(cum, g, off);
        // segment k of row task L: the last one starting at or before off
        // (an empty segment shares its start with the next one)
        const int4 ss = sh.sst[L];
        const int k = (off >= ss.x) + (off >= ss.y) + (off >= ss.z);
        off -= k == 0 ? 0 : k == 1 ? ss.x : k == 2 ? ss.y : ss.z;
        const float4 sg = sh.seg[L * 4 + k];
        const int X = __float_as_int(sg.w) + off;
        const float a = sg.z * mean2_clamp01f(sg.x - (float)X, sg.y - (float)X);
        if (a != 0.0f) {
          const int2 rb = sh.rbi[L];
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
}

}  // namespace
}  // namespace lens
