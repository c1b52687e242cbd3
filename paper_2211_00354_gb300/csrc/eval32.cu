// eval32.cu -- the float32-bulk form of the fused per-ray FMM evaluation
// (L2P, Appendix A step 6; P2P with the adjacent leaves, step 7; M2P for
// the adaptive W lists; the lens equation, Eq. 1 with kappa_s and gamma).
//
// GB300's float64 pipe issues ~2 lanes per clock per SM, so a warp-wide
// float64 instruction costs ~16 issue cycles: even per-CTA float64 set-up
// (leaf centre, offsets of staged stars) executed by every thread rivals the
// float32 pair work.  This kernel therefore runs no float64 instruction at
// all on the grid path.  Everything float64 is done once:
//   per plan  -- float32 copies of the local (L) and multipole (M)
//                coefficients; every active leaf's near-field stars (its
//                U-list leaves and the W boxes with at most (p+1)/2 stars,
//                for which a direct sum is cheaper than an order-p M2P) as
//                float-float offsets from the leaf centre plus float32
//                masses; the remaining W boxes' centre offsets and radii in
//                float32; per-leaf
//                constants K1 = a c1 - b0_1, K2 = b c2 + b0_2 (the lens
//                equation evaluated at the centre with the constant term b0
//                of the local expansion), 1/r;
//   per call  -- per leaf, the float-float offset of its first grid ray from
//                the centre and (map path) the leaf's pixel reference point.
// Per ray: offset dx = (x(i0) - c) + (i - i0) h in float-float; near field
// d = (x_hi - s_hi) + (x_lo - s_lo) summed per source leaf in float32 and
// accumulated by two-sum; L2P/M2P by Horner in float32; then
//   y1 = K1 + (a dx - f1 - near1),  y2 = K2 + (b dy + f2 - near2)
// with the bracket in float-float (alpha = conj(b0 + f + near)).  On the map
// path the corner goes straight to pixel coordinates u = U1 + (y1 - K1)/du,
// split into an integer pixel and a float32 fraction for the IPM kernels.
#include <algorithm>
#include <vector>

#include "cx.cuh"
#include "ipm_warp.cuh"
#include "lens_internal.h"

namespace lens {

namespace {

constexpr int kT = kEval32Threads;
constexpr int kRpt = kEval32Rpt;
constexpr int kGroup = 8;  // stars per float32 partial sum of the near field
constexpr int kChunk = 512;
static_assert(kRpt % 2 == 0, "rays are paired for float2 arithmetic");
constexpr int kWChunk = 8;

struct E32Args {
  const LeafPlan* leaf;
  const int* leaves;
  const int2* tile_leaf;  // (leaf, tile within the leaf) of each block
  int64_t nleaf;
  const int* aidx;
  const int* count;
  // per active leaf k: its near-field stars (U-list leaves and small W
  // boxes, P2P) staged at ust/um[uoff[k] .. uoff[k+1]); far W boxes (M2P)
  // wlist[woff[k] .. woff[k+1])
  const int64_t* woff; const int* wlist;
  const float2* fL; const float2* fM;
  const float4* ust; const float* um; const int64_t* uoff; const float4* wgeo;
  int p;
  ff af, bf;
  bool unit_mass;  // every star has mass m0 (near field summed without the mass)
  float m0;
  double a, b;
  // grid source
  const int64_t* rect; const LeafGrid* lgrid; ff hf; int64_t gnx1, grow0;
  ff ihf;  // 1 / h: the grid path's near field runs in grid units
  // ray source
  const double* rays; const int64_t* ray_off; const int* perm;
  double* y; double* jac;
  PixCorner* pix; ff iduf, idvf;
};

// Shared memory of the float32 evaluation: the staged near stars, each value
// duplicated into both halves of a float2 (the offsets negated, so that
// d = x + (-s) is the plain difference), and the expansion coefficients with
// each real / imaginary part duplicated (operands of the paired-ray
// arithmetic).
struct E32Smem {
  float2 s_x[kChunk], s_y[kChunk], s_xl[kChunk], s_yl[kChunk], s_m[kChunk];
  float2 s_Lx[kMaxOrder + 1], s_Ly[kMaxOrder + 1];
  float2 s_Wx[kWChunk][kMaxOrder + 1], s_Wy[kWChunk][kMaxOrder + 1];
  float4 s_wg[kWChunk];
};

// The leaf's float32 local coefficients (block-cooperative; a barrier must
// follow before they are read).
__device__ __forceinline__ void stage_local(E32Smem& sm, const E32Args& A, int64_t k, int tid) {
  const int p = A.p;
  for (int l = tid; l <= p; l += kT) {
    const float2 c = A.fL[k * (int64_t)(p + 1) + l];
    sm.s_Lx[l] = make_float2(c.x, c.x);
    sm.s_Ly[l] = make_float2(c.y, c.y);
  }
}

// Near stars g0 .. g0 + nf - 1 of a leaf into the staging arrays, padded to nfg
// (whole groups of kGroup) with massless stars 1e18 away: they add exactly
// zero when the mass multiplies (w = 0 * finite) and ~1e-18 (far below
// float32 rounding of the sum) in the equal-mass form, which leaves the mass
// out.  Block-cooperative, between barriers.
//
// On the grid path (GU) the stars are staged in grid units relative to the
// leaf's grid origin instead: sigma = (s - x_o) / h as float-float (bx, by:
// the origin's offset from the leaf centre), so that a ray's own coordinates
// are integers and a difference is (i - sigma_hi) - sigma_lo, two roundings
// like the float-float form.
template <bool GU>
__device__ __forceinline__ void stage_stars(E32Smem& sm, const E32Args& A, int64_t g0, int nf,
                                            int nfg, int tid, ff bx = ff{0.f, 0.f},
                                            ff by = ff{0.f, 0.f}) {
  for (int f = tid; f < nfg; f += kT) {
    float4 v = make_float4(1e18f, 0.f, 0.f, 0.f);
    float mm = 0.f;
    if (f < nf) {
      v = A.ust[g0 + f];
      mm = A.um[g0 + f];
    }
    if (GU) {
      const ff gx = ff_mul(ff_add(ff{v.x, v.z}, ff_neg(bx)), A.ihf);
      const ff gy = ff_mul(ff_add(ff{v.y, v.w}, ff_neg(by)), A.ihf);
      v = make_float4(gx.hi, gy.hi, gx.lo, gy.lo);
    }
    sm.s_x[f] = make_float2(-v.x, -v.x); sm.s_y[f] = make_float2(-v.y, -v.y);
    sm.s_xl[f] = make_float2(-v.z, -v.z); sm.s_yl[f] = make_float2(-v.w, -v.w);
    sm.s_m[f] = make_float2(mm, mm);
  }
}

// P2P of a thread's rays against the nfg staged stars, rays (2h, 2h+1) side
// by side in float2 pair arithmetic (Blackwell's two-lane FP32 instructions,
// IEEE round-to-nearest per lane): summed in groups of kGroup stars in plain
// float32, each group partial entering the two-sum accumulators N1, N2.  A
// star exactly on the ray contributes nothing: the floor on r2 keeps w
// finite and w * d = 0.
// GU: grid units, the rays' coordinates exact integers in dx, dy (dxl, dyl
// unused): d = (x - s_hi) - s_lo, one paired add fewer per coordinate.  A
// padding star then lies ~1e18 / h away: its |d|^2 may overflow to infinity,
// whose reciprocal 0 still makes its term exactly zero.
template <bool UM, bool GU = false>
__device__ __forceinline__ void p2p_paired(const E32Smem& sm, int nfg, const float (&dx)[kRpt],
                                           const float (&dy)[kRpt], const float (&dxl)[kRpt],
                                           const float (&dyl)[kRpt], fcomp2 (&N1)[kRpt / 2],
                                           fcomp2 (&N2)[kRpt / 2]) {
  for (int lo = 0; lo < nfg; lo += kGroup) {
    float2 P1[kRpt / 2], P2[kRpt / 2], DX[kRpt / 2], DY[kRpt / 2], DXL[kRpt / 2], DYL[kRpt / 2];
#pragma unroll
    for (int h = 0; h < kRpt / 2; ++h) {
      P1[h] = make_float2(0.f, 0.f); P2[h] = make_float2(0.f, 0.f);
      DX[h] = make_float2(dx[2 * h], dx[2 * h + 1]); DY[h] = make_float2(dy[2 * h], dy[2 * h + 1]);
      DXL[h] = make_float2(dxl[2 * h], dxl[2 * h + 1]); DYL[h] = make_float2(dyl[2 * h], dyl[2 * h + 1]);
    }
    const float2 tiny = make_float2(1e-30f, 1e-30f);
#pragma unroll
    for (int jj = 0; jj < kGroup; ++jj) {
      const int j = lo + jj;
      const float2 nsx = sm.s_x[j], nsy = sm.s_y[j], nsxl = sm.s_xl[j], nsyl = sm.s_yl[j];
#pragma unroll
      for (int h = 0; h < kRpt / 2; ++h) {
        const float2 d1 = GU ? __fadd2_rn(__fadd2_rn(DX[h], nsx), nsxl)
                             : __fadd2_rn(__fadd2_rn(DX[h], nsx), __fadd2_rn(DXL[h], nsxl));
        const float2 d2 = GU ? __fadd2_rn(__fadd2_rn(DY[h], nsy), nsyl)
                             : __fadd2_rn(__fadd2_rn(DY[h], nsy), __fadd2_rn(DYL[h], nsyl));
        const float2 r2 = __ffma2_rn(d1, d1, __ffma2_rn(d2, d2, tiny));
        const float2 rr = make_float2(frcp_fast(r2.x), frcp_fast(r2.y));
        // equal masses: the mass multiplies the sums once, after the loop
        const float2 w = UM ? rr : __fmul2_rn(sm.s_m[j], rr);
        P1[h] = __ffma2_rn(w, d1, P1[h]);
        P2[h] = __ffma2_rn(w, d2, P2[h]);
      }
    }
#pragma unroll
    for (int h = 0; h < kRpt / 2; ++h) {
      N1[h].add(P1[h]);
      N2[h].add(P2[h]);
    }
  }
}

// far W boxes e0 .. e0 + nw - 1 of a leaf (their float32 multipoles and
// geometry) into shared memory; block-cooperative, between barriers
__device__ __forceinline__ void stage_w(E32Smem& sm, const E32Args& A, int64_t e0, int nw, int tid) {
  const int p = A.p;
  for (int t = tid; t < nw * (p + 1); t += kT) {
    const int w = t / (p + 1), kk = t - w * (p + 1);
    const float2 c = A.fM[(int64_t)A.wlist[e0 + w] * (p + 1) + kk];
    sm.s_Wx[w][kk] = make_float2(c.x, c.x);
    sm.s_Wy[w][kk] = make_float2(c.y, c.y);
  }
  if (tid < nw) sm.s_wg[tid] = A.wgeo[e0 + tid];
}

// M2P of the nw staged W boxes, rays (2h, 2h+1) side by side: Horner's rule
// for f(z) = (1/z) sum_k A_k (r/z)^k, 4 paired multiply-adds per order.
__device__ __forceinline__ void m2p_paired(const E32Smem& sm, int nw, int p, const float (&dx)[kRpt],
                                           const float (&dy)[kRpt], float2 (&FX)[kRpt / 2],
                                           float2 (&FY)[kRpt / 2]) {
  for (int w = 0; w < nw; ++w) {
    const float4 gw = sm.s_wg[w];
    const float2 ngx = make_float2(-gw.x, -gw.x), ngy = make_float2(-gw.y, -gw.y);
    const float2 gr = make_float2(gw.z, gw.z), ngr = make_float2(-gw.z, -gw.z);
#pragma unroll
    for (int h = 0; h < kRpt / 2; ++h) {
      const float2 zx = __fadd2_rn(make_float2(dx[2 * h], dx[2 * h + 1]), ngx);
      const float2 zy = __fadd2_rn(make_float2(dy[2 * h], dy[2 * h + 1]), ngy);
      const float2 n2 = __ffma2_rn(zx, zx, __fmul2_rn(zy, zy));
      const float2 d = make_float2(frcp_fast(n2.x), frcp_fast(n2.y));
      const float2 ix = __fmul2_rn(zx, d);   // 1/z = (zx d, -zy d)
      const float2 niy = __fmul2_rn(zy, d);  // -Im(1/z)
      const float2 iy = make_float2(-niy.x, -niy.y);
      const float2 qx = __fmul2_rn(ix, gr), qy = __fmul2_rn(iy, gr);
      const float2 nqy = __fmul2_rn(iy, ngr);
      float2 sx = sm.s_Wx[w][p], sy = sm.s_Wy[w][p];
      for (int kk = p - 1; kk >= 0; --kk) {
        const float2 tx = __ffma2_rn(sy, nqy, sm.s_Wx[w][kk]);
        const float2 ty = __ffma2_rn(sy, qx, sm.s_Wy[w][kk]);
        const float2 nsx = __ffma2_rn(sx, qx, tx);
        sy = __ffma2_rn(sx, qy, ty);
        sx = nsx;
      }
      FX[h] = __ffma2_rn(sx, ix, __ffma2_rn(sy, niy, FX[h]));
      FY[h] = __ffma2_rn(sx, iy, __ffma2_rn(sy, ix, FY[h]));
    }
  }
}

// L2P by Horner's rule and the float-float lens equation for rays (2h, 2h+1)
// side by side: T1 = a dx - Re f - near1, T2 = b dy + Im f - near2 (y minus
// the leaf's float64 constant; alpha = conj(b0 + f + near)).
// (GU: the near-field sums are in grid units and take the factor 1/h here.)
template <bool GU = false>
__device__ __forceinline__ void l2p_lens_pair(const E32Smem& sm, const E32Args& A, float ir, int h,
                                              const float (&dx)[kRpt], const float (&dy)[kRpt],
                                              const float (&dxl)[kRpt], const float (&dyl)[kRpt],
                                              const fcomp2& N1h, const fcomp2& N2h, float2 FXh,
                                              float2 FYh, ff2& T1, ff2& T2) {
  const int p = A.p;
  const float2 irr = make_float2(ir, ir), nirr = make_float2(-ir, -ir);
  const float2 DXh = make_float2(dx[2 * h], dx[2 * h + 1]);
  const float2 DYh = make_float2(dy[2 * h], dy[2 * h + 1]);
  const float2 wx = __fmul2_rn(DXh, irr);
  const float2 wy = __fmul2_rn(DYh, irr);
  const float2 nwy = __fmul2_rn(DYh, nirr);
  float2 fx = make_float2(0.f, 0.f), fy = make_float2(0.f, 0.f);
  if (p >= 1) {
    float2 sx = sm.s_Lx[p], sy = sm.s_Ly[p];
    for (int l = p - 1; l >= 1; --l) {
      const float2 tx = __ffma2_rn(sy, nwy, sm.s_Lx[l]);
      const float2 ty = __ffma2_rn(sy, wx, sm.s_Ly[l]);
      const float2 nsx = __ffma2_rn(sx, wx, tx);
      sy = __ffma2_rn(sx, wy, ty);
      sx = nsx;
    }
    fx = __ffma2_rn(sx, wx, __fmul2_rn(sy, nwy));
    fy = __ffma2_rn(sx, wy, __fmul2_rn(sy, wx));
  }
  // f = L2P + M2P (the far W boxes)
  fx = __fadd2_rn(fx, FXh);
  fy = __fadd2_rn(fy, FYh);
  // y1 = a x1 - Re f - near1, y2 = b x2 + Im f - near2 (alpha = conj f)
  const ff2 n1 = GU ? ff2_mul(A.ihf, ff2{N1h.hi, N1h.lo}) : ff2{N1h.hi, N1h.lo};
  const ff2 n2 = GU ? ff2_mul(A.ihf, ff2{N2h.hi, N2h.lo}) : ff2{N2h.hi, N2h.lo};
  T1 = ff2_mul(A.af, ff2{DXh, make_float2(dxl[2 * h], dxl[2 * h + 1])});
  T1 = ff2_sub(T1, fx);
  T1 = ff2_sub(T1, n1);
  T2 = ff2_mul(A.bf, ff2{DYh, make_float2(dyl[2 * h], dyl[2 * h + 1])});
  T2 = ff2_add(T2, fy);
  T2 = ff2_sub(T2, n2);
}

// The two rays' source-plane positions in map-pixel coordinates: u = U1 +
// T1 / du (U1 the leaf centre's reference), split into an integer pixel and a
// float32 fraction in [0, 1); corners beyond 2^30 pixels are marked far.
__device__ __forceinline__ void pix_pair(const E32Args& A, const LeafGrid& lg, const ff2& T1,
                                         const ff2& T2, PixCorner (&pc)[2]) {
  const ff2 U = ff2_add(lg.U1f, ff2_mul(A.iduf, T1));
  const ff2 V = ff2_add(lg.V1f, ff2_mul(A.idvf, T2));
  const float2 ku2 = make_float2(floorf(U.hi.x), floorf(U.hi.y));
  const float2 kv2 = make_float2(floorf(V.hi.x), floorf(V.hi.y));
  const float2 fu2 = __fadd2_rn(fsub2(U.hi, ku2), U.lo);
  const float2 fv2 = __fadd2_rn(fsub2(V.hi, kv2), V.lo);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const float uh = c ? U.hi.y : U.hi.x, vh = c ? V.hi.y : V.hi.x;
    float ku = c ? ku2.y : ku2.x, kv = c ? kv2.y : kv2.x;
    float fu = c ? fu2.y : fu2.x, fv = c ? fv2.y : fv2.x;
    bool far = lg.far || !(fabsf(uh) < 5.0e8f) || !(fabsf(vh) < 5.0e8f);
    if (fu < 0.f) { ku -= 1.f; fu += 1.f; } else if (fu >= 1.f) { ku += 1.f; fu -= 1.f; }
    if (fv < 0.f) { kv -= 1.f; fv += 1.f; } else if (fv >= 1.f) { kv += 1.f; fv -= 1.f; }
    // float -> int32 (|k| < 5e8); integer adds only afterwards
    const int64_t iu = (int64_t)lg.U1i + (int)ku, iv = (int64_t)lg.V1i + (int)kv;
    far = far || !(iu > -1073741824ll && iu < 1073741824ll && iv > -1073741824ll &&
                   iv < 1073741824ll);
    if (!far) {
      pc[c].iu = (int)iu; pc[c].fu = fu; pc[c].iv = (int)iv; pc[c].fv = fv;
    } else {
      pc[c].iu = 0x7fffffff; pc[c].fu = 0.f; pc[c].iv = 0x7fffffff; pc[c].fv = 0.f;
    }
  }
}

// The offset of grid ray (di, dj) of a leaf (counted from the leaf's first
// ray) from the leaf centre, float-float; int32 -> float only (64-bit forms
// run on the float64 pipe).
__device__ __forceinline__ void grid_offset(const E32Args& A, const LeafGrid& lg, uint32_t di,
                                            uint32_t dj, float& dx, float& dxl, float& dy,
                                            float& dyl) {
  const ff ox = ff_add(lg.bx, ff_mul(A.hf, (float)(int)di));
  const ff oy = ff_add(lg.by, ff_mul(A.hf, (float)(int)dj));
  dx = ox.hi; dxl = ox.lo;
  dy = oy.hi; dyl = oy.lo;
}

template <bool JAC, bool GRID, bool PIX, bool UM = false>
__global__ void __launch_bounds__(kT, 7) k_eval32(E32Args A) {
  __shared__ E32Smem sm;
  const int tid = threadIdx.x;
  const int p = A.p;
  const int2 kt = A.tile_leaf[blockIdx.x];
  const int64_t k = kt.x;
  const int64_t tile = kt.y;
  const LeafPlan lp = A.leaf[k];
  stage_local(sm, A, k, tid);

  // ---- rays of this tile -------------------------------------------------
  int64_t nr_leaf, i0 = 0, ni = 1, j0 = 0;
  LeafGrid lg{};
  if (GRID) {
    i0 = A.rect[4 * k]; ni = A.rect[4 * k + 1]; j0 = A.rect[4 * k + 2];
    nr_leaf = ni * A.rect[4 * k + 3];
    lg = A.lgrid[k];
  } else {
    nr_leaf = A.ray_off[k + 1] - A.ray_off[k];
  }
  // the grid path without the Jacobian sums its near field in grid units
  constexpr bool GU = GRID && !JAC;
  float dx[kRpt], dy[kRpt], dxl[kRpt], dyl[kRpt];
  float gxr[kRpt], gyr[kRpt];  // GU: the rays' integer grid coordinates from the leaf's origin
  int64_t oidx[kRpt];
  bool ok[kRpt];
  fcomp n1[kRpt], n2[kRpt], nj1[kRpt], nj2[kRpt];
  fcomp2 N1[kRpt / 2], N2[kRpt / 2];  // paired accumulators of the Jacobian-free path
#pragma unroll
  for (int h = 0; h < kRpt / 2; ++h) {
    N1[h] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    N2[h] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  }
  // A tile holds up to kT kRpt rays; a partial one (a leaf's last tile, or a
  // leaf of few rays) lays them out with stride S, a multiple of 32, so that
  // they fill whole warps: slot q of thread t is ray q S + t of the tile, and a
  // warp with no ray (t >= S) joins the block's staging but skips the sums.
  const int64_t tbase = tile * (int64_t)(kT * kRpt);
  const int nt = (int)min64(kT * kRpt, nr_leaf - tbase);
  const int S = min(kT, ((nt + kRpt - 1) / kRpt + 31) & ~31);
  const bool live = (tid & ~31) < S;
#pragma unroll
  for (int q = 0; q < kRpt; ++q) {
    const int64_t loc = tbase + (int64_t)q * S + tid;
    ok[q] = tid < S && loc < nr_leaf;
    dx[q] = dy[q] = dxl[q] = dyl[q] = 0.f;
    gxr[q] = gyr[q] = 0.f;
    oidx[q] = 0;
    n1[q] = {0.f, 0.f}; n2[q] = {0.f, 0.f}; nj1[q] = {0.f, 0.f}; nj2[q] = {0.f, 0.f};
    if (!ok[q]) continue;
    if (GRID) {
      // 32-bit division
      const uint32_t l32 = (uint32_t)loc, n32 = (uint32_t)ni;
      const uint32_t dj = l32 / n32, di = l32 - dj * n32;
      oidx[q] = (j0 + (int64_t)dj - A.grow0) * A.gnx1 + i0 + (int64_t)di;
      grid_offset(A, lg, di, dj, dx[q], dxl[q], dy[q], dyl[q]);
      gxr[q] = (float)(lg.ri + (int)di);
      gyr[q] = (float)(lg.rj + (int)dj);
    } else {
      const int64_t ridx = A.perm[A.ray_off[k] + loc];
      oidx[q] = ridx;
      const double ox = A.rays[2 * ridx] - lp.cx, oy = A.rays[2 * ridx + 1] - lp.cy;
      dx[q] = (float)ox; dxl[q] = (float)(ox - (double)dx[q]);
      dy[q] = (float)oy; dyl[q] = (float)(oy - (double)dy[q]);
    }
  }

  // ---- P2P over the near field (stars pre-staged per leaf in float-float) --
  // The leaf's near stars are contiguous: they are staged kChunk at a time
  // and summed in groups of kGroup (8) in plain float32, each group partial then
  // entering a two-sum (compensated) accumulator.  The staged chunk is padded
  // to whole groups, so every group loop has a fixed trip count and unrolls.
  static_assert(kChunk % kGroup == 0, "chunks hold whole groups");
  const int64_t star0 = A.uoff[k], nstar = A.uoff[k + 1] - star0;
  for (int64_t f0 = 0; f0 < nstar; f0 += kChunk) {
    const int nf = (int)min64(kChunk, nstar - f0);
    const int nfg = (nf + kGroup - 1) / kGroup * kGroup;
    __syncthreads();
    stage_stars<GU>(sm, A, star0 + f0, nf, nfg, tid, lg.rx, lg.ry);
    __syncthreads();
    if (!live) continue;  // uniform over the warp; the barriers are above
    if constexpr (GU) {
      p2p_paired<UM, true>(sm, nfg, gxr, gyr, dxl, dyl, N1, N2);
    } else if (!JAC) {
      p2p_paired<UM>(sm, nfg, dx, dy, dxl, dyl, N1, N2);
    } else {
      for (int lo = 0; lo < nfg; lo += kGroup) {
        float p1[kRpt], p2[kRpt], pj1[kRpt], pj2[kRpt];
#pragma unroll
        for (int q = 0; q < kRpt; ++q) { p1[q] = 0.f; p2[q] = 0.f; pj1[q] = 0.f; pj2[q] = 0.f; }
#pragma unroll
        for (int jj = 0; jj < kGroup; ++jj) {
          const int j = lo + jj;
          const float sx = -sm.s_x[j].x, sy = -sm.s_y[j].x, sxl = -sm.s_xl[j].x, syl = -sm.s_yl[j].x;
          const float smm = sm.s_m[j].x;
#pragma unroll
          for (int q = 0; q < kRpt; ++q) {
            const float d1 = (dx[q] - sx) + (dxl[q] - sxl);
            const float d2 = (dy[q] - sy) + (dyl[q] - syl);
            // a star exactly on the ray contributes nothing (w * w would
            // overflow with a floor on r2, hence the select)
            const float r2 = fmaf(d1, d1, d2 * d2);
            const float inv = r2 > 0.f ? frcp_fast(r2) : 0.f;
            const float w = smm * inv;
            p1[q] = fmaf(w, d1, p1[q]);
            p2[q] = fmaf(w, d2, p2[q]);
            const float w2 = w * inv;
            pj1[q] = fmaf(w2, (d2 - d1) * (d2 + d1), pj1[q]);
            pj2[q] = fmaf(w2, 2.f * d1 * d2, pj2[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < kRpt; ++q) {
          n1[q].add(p1[q]); n2[q].add(p2[q]);
          nj1[q].add(pj1[q]); nj2[q].add(pj2[q]);
        }
      }
    }
  }

  if constexpr (!JAC && UM) {
    if (A.m0 != 1.f) {
      const float2 m2 = make_float2(A.m0, A.m0);
#pragma unroll
      for (int h = 0; h < kRpt / 2; ++h) {
        N1[h].hi = __fmul2_rn(N1[h].hi, m2); N1[h].lo = __fmul2_rn(N1[h].lo, m2);
        N2[h].hi = __fmul2_rn(N2[h].hi, m2); N2[h].lo = __fmul2_rn(N2[h].lo, m2);
      }
    }
  }

  // ---- M2P over the far W boxes --------------------------------------------
  float2 fw[kRpt], dfw[kRpt];
#pragma unroll
  for (int q = 0; q < kRpt; ++q) { fw[q] = make_float2(0.f, 0.f); dfw[q] = make_float2(0.f, 0.f); }
  float2 FX[kRpt / 2], FY[kRpt / 2];
#pragma unroll
  for (int h = 0; h < kRpt / 2; ++h) { FX[h] = make_float2(0.f, 0.f); FY[h] = make_float2(0.f, 0.f); }
  const int64_t w_beg = A.woff[k], w_end = A.woff[k + 1];
  for (int64_t e0 = w_beg; e0 < w_end; e0 += kWChunk) {
    const int nw = (int)min64(kWChunk, w_end - e0);
    __syncthreads();
    stage_w(sm, A, e0, nw, tid);
    __syncthreads();
    if (!live) continue;
    if (!JAC) {
      m2p_paired(sm, nw, p, dx, dy, FX, FY);
    } else {
      for (int w = 0; w < nw; ++w) {
        const float4 gw = sm.s_wg[w];
#pragma unroll
        for (int q = 0; q < kRpt; ++q) {
          const float2 z = make_float2(dx[q] - gw.x, dy[q] - gw.y);
          const float2 inv = cinv(z);
          const float2 qq = make_float2(inv.x * gw.z, inv.y * gw.z);
          float2 s = make_float2(sm.s_Wx[w][p].x, sm.s_Wy[w][p].x);
          for (int kk = p - 1; kk >= 0; --kk) s = cfma(s, qq, make_float2(sm.s_Wx[w][kk].x, sm.s_Wy[w][kk].x));
          fw[q] = cfma(s, inv, fw[q]);
          float2 t = make_float2((float)(p + 1) * sm.s_Wx[w][p].x, (float)(p + 1) * sm.s_Wy[w][p].x);
          for (int kk = p - 1; kk >= 0; --kk)
            t = cfma(t, qq, make_float2((float)(kk + 1) * sm.s_Wx[w][kk].x, (float)(kk + 1) * sm.s_Wy[w][kk].x));
          const float2 dd = cmul(t, cmul(inv, inv));
          dfw[q] = make_float2(dfw[q].x - dd.x, dfw[q].y - dd.y);
        }
      }
    }
  }

  // ---- L2P + epilogue --------------------------------------------------------
  __syncthreads();
  if (!live) return;  // no barrier follows
  const float ir = lp.ir;
  if constexpr (!JAC) {
#pragma unroll
    for (int h = 0; h < kRpt / 2; ++h) {
      ff2 T1, T2;
      l2p_lens_pair<GU>(sm, A, ir, h, dx, dy, dxl, dyl, N1[h], N2[h], FX[h], FY[h], T1, T2);
      if (PIX) {
        PixCorner pc[2];
        pix_pair(A, lg, T1, T2, pc);
        if (ok[2 * h]) A.pix[oidx[2 * h]] = pc[0];
        if (ok[2 * h + 1]) A.pix[oidx[2 * h + 1]] = pc[1];
      } else {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int q = 2 * h + c;
          if (!ok[q]) continue;
          const ff t1 = c ? ff{T1.hi.y, T1.lo.y} : ff{T1.hi.x, T1.lo.x};
          const ff t2 = c ? ff{T2.hi.y, T2.lo.y} : ff{T2.hi.x, T2.lo.x};
          A.y[2 * oidx[q]] = lp.K1 + ff_to_double(t1);
          A.y[2 * oidx[q] + 1] = lp.K2 + ff_to_double(t2);
        }
      }
    }
  } else {
    // with the Jacobian: one ray at a time
#pragma unroll
    for (int q = 0; q < kRpt; ++q) {
      if (!ok[q]) continue;
      float2 f = make_float2(0.f, 0.f), df = make_float2(0.f, 0.f);
      if (p >= 1) {
        const float2 w = make_float2(dx[q] * ir, dy[q] * ir);
        float2 s = make_float2(sm.s_Lx[p].x, sm.s_Ly[p].x);
        for (int l = p - 1; l >= 1; --l) s = cfma(s, w, make_float2(sm.s_Lx[l].x, sm.s_Ly[l].x));
        f = cmul(s, w);
        float2 t = make_float2((float)p * sm.s_Lx[p].x, (float)p * sm.s_Ly[p].x);
        for (int l = p - 1; l >= 1; --l)
          t = cfma(t, w, make_float2((float)l * sm.s_Lx[l].x, (float)l * sm.s_Ly[l].x));
        df = make_float2(t.x * ir, t.y * ir);
      }
      f = f + fw[q];
      ff T1 = ff_mul(A.af, ff{dx[q], dxl[q]});
      T1 = ff_add(T1, -f.x);
      T1 = ff_add(T1, ff{-n1[q].hi, -n1[q].lo});
      ff T2 = ff_mul(A.bf, ff{dy[q], dyl[q]});
      T2 = ff_add(T2, f.y);
      T2 = ff_add(T2, ff{-n2[q].hi, -n2[q].lo});
      if (PIX) {
        PixCorner pc;
        const ff U = ff_add(lg.U1f, ff_mul(A.iduf, T1));
        const ff V = ff_add(lg.V1f, ff_mul(A.idvf, T2));
        bool far = lg.far || !(fabsf(U.hi) < 5.0e8f) || !(fabsf(V.hi) < 5.0e8f);
        float ku = floorf(U.hi), kv = floorf(V.hi);
        float fu = (U.hi - ku) + U.lo, fv = (V.hi - kv) + V.lo;
        if (fu < 0.f) { ku -= 1.f; fu += 1.f; } else if (fu >= 1.f) { ku += 1.f; fu -= 1.f; }
        if (fv < 0.f) { kv -= 1.f; fv += 1.f; } else if (fv >= 1.f) { kv += 1.f; fv -= 1.f; }
        // float -> int32 (|k| < 5e8); integer adds only afterwards
        const int64_t iu = (int64_t)lg.U1i + (int)ku, iv = (int64_t)lg.V1i + (int)kv;
        far = far || !(iu > -1073741824ll && iu < 1073741824ll && iv > -1073741824ll &&
                       iv < 1073741824ll);
        if (!far) {
          pc.iu = (int)iu; pc.fu = fu; pc.iv = (int)iv; pc.fv = fv;
        } else {
          pc.iu = 0x7fffffff; pc.fu = 0.f; pc.iv = 0x7fffffff; pc.fv = 0.f;
        }
        A.pix[oidx[q]] = pc;
        continue;
      }
      A.y[2 * oidx[q]] = lp.K1 + ff_to_double(T1);
      A.y[2 * oidx[q] + 1] = lp.K2 + ff_to_double(T2);
      if (JAC) {
        const double dre = (double)df.x + (double)dfw[q].x + nj1[q].value();
        const double dim = (double)df.y + (double)dfw[q].y + nj2[q].value();
        A.jac[4 * oidx[q] + 0] = A.a - dre;
        A.jac[4 * oidx[q] + 1] = dim;
        A.jac[4 * oidx[q] + 2] = dim;
        A.jac[4 * oidx[q] + 3] = A.b + dre;
      }
    }
  }
}

// ---- fused deflection + IPM (Sec. 2.4 steps 3-4 without a corner array) --
// A block takes one work item (FuseItem: a rectangle of one leaf's grid
// corners).  It evaluates the item's corners exactly as k_eval32 does (the
// same leaf data, the same operations: a corner that two items of the leaf
// share gets the same bits from both), keeps them in shared memory as pixel
// coordinates, writes only those on the leaf's first or last corner row or
// column to `edge`, and then maps every cell whose four corners lie in the
// item with the warp IPM of k_ipm_cells (ill-conditioned cells by the whole
// warp on the spot).  Cells on the leaf's last corner row or column are left
// to the seam pass.
constexpr int kFuseCorners = 1024;  // corners per item: two groups of kT x kRpt rays
constexpr int kFuseSeg = 128;       // corner columns per item at most
constexpr int kFuseWarps = kT / 32;

template <bool UM>
__global__ void __launch_bounds__(kT, 4) k_eval32_map(E32Args A, IpmArgs I, const FuseItem* items,
                                                   PixCorner* edge) {
  // the evaluation's staging and the IPM's per-warp staging are used one
  // after the other
  __shared__ union Stage {
    E32Smem e;
    struct {
      WarpCells c[kFuseWarps];
      int cut[kFuseWarps][128];  // cut pixels of the warp's float-float cell
    } m;
  } sm;
  __shared__ PixCorner cs[kFuseCorners];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const FuseItem it = items[blockIdx.x];
  const int64_t k = it.leaf;
  const LeafGrid lg = A.lgrid[k];
  const int64_t i0 = A.rect[4 * k], ni = A.rect[4 * k + 1];
  const int64_t j0 = A.rect[4 * k + 2], nj = A.rect[4 * k + 3];
  const float ir = A.leaf[k].ir;
  stage_local(sm.e, A, k, tid);
  const int ncorn = it.w * it.h;
  const int ngroups = (ncorn + kT * kRpt - 1) / (kT * kRpt);
  const int64_t star0 = A.uoff[k], nstar = A.uoff[k + 1] - star0;
  const int64_t w_beg = A.woff[k], w_end = A.woff[k + 1];
  // a leaf whose near stars (W boxes) fill one staging chunk stages them once
  const bool restage_stars = nstar > kChunk, restage_w = w_end - w_beg > kWChunk;
  for (int g = 0; g < ngroups; ++g) {
    float dx[kRpt], dy[kRpt], dxl[kRpt], dyl[kRpt];
    float gxr[kRpt], gyr[kRpt];  // the rays' integer grid coordinates from the leaf's origin
    int t[kRpt];
    bool ok[kRpt];
    uint32_t di[kRpt], dj[kRpt];
    fcomp2 N1[kRpt / 2], N2[kRpt / 2];
#pragma unroll
    for (int h = 0; h < kRpt / 2; ++h) {
      N1[h] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      N2[h] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
#pragma unroll
    for (int q = 0; q < kRpt; ++q) {
      t[q] = g * (kT * kRpt) + q * kT + tid;
      ok[q] = t[q] < ncorn;
      dx[q] = dy[q] = dxl[q] = dyl[q] = 0.f;
      gxr[q] = gyr[q] = 0.f;
      di[q] = dj[q] = 0;
      if (!ok[q]) continue;
      const uint32_t r = (uint32_t)t[q] / (uint32_t)it.w, c = (uint32_t)t[q] - r * (uint32_t)it.w;
      di[q] = (uint32_t)it.ci + c;
      dj[q] = (uint32_t)it.cj + r;
      grid_offset(A, lg, di[q], dj[q], dx[q], dxl[q], dy[q], dyl[q]);
      gxr[q] = (float)(lg.ri + (int)di[q]);
      gyr[q] = (float)(lg.rj + (int)dj[q]);
    }
    for (int64_t f0 = 0; f0 < nstar; f0 += kChunk) {
      const int nf = (int)min64(kChunk, nstar - f0);
      const int nfg = (nf + kGroup - 1) / kGroup * kGroup;
      if (g == 0 || restage_stars) {
        __syncthreads();
        stage_stars<true>(sm.e, A, star0 + f0, nf, nfg, tid, lg.rx, lg.ry);
        __syncthreads();
      }
      p2p_paired<UM, true>(sm.e, nfg, gxr, gyr, dxl, dyl, N1, N2);
    }
    if (UM && A.m0 != 1.f) {
      const float2 m2 = make_float2(A.m0, A.m0);
#pragma unroll
      for (int h = 0; h < kRpt / 2; ++h) {
        N1[h].hi = __fmul2_rn(N1[h].hi, m2); N1[h].lo = __fmul2_rn(N1[h].lo, m2);
        N2[h].hi = __fmul2_rn(N2[h].hi, m2); N2[h].lo = __fmul2_rn(N2[h].lo, m2);
      }
    }
    float2 FX[kRpt / 2], FY[kRpt / 2];
#pragma unroll
    for (int h = 0; h < kRpt / 2; ++h) { FX[h] = make_float2(0.f, 0.f); FY[h] = make_float2(0.f, 0.f); }
    for (int64_t e0 = w_beg; e0 < w_end; e0 += kWChunk) {
      const int nw = (int)min64(kWChunk, w_end - e0);
      if (g == 0 || restage_w) {
        __syncthreads();
        stage_w(sm.e, A, e0, nw, tid);
        __syncthreads();
      }
      m2p_paired(sm.e, nw, A.p, dx, dy, FX, FY);
    }
    if (g == 0) __syncthreads();  // the local coefficients, with no star or W chunk staged
#pragma unroll
    for (int h = 0; h < kRpt / 2; ++h) {
      ff2 T1, T2;
      l2p_lens_pair<true>(sm.e, A, ir, h, dx, dy, dxl, dyl, N1[h], N2[h], FX[h], FY[h], T1, T2);
      PixCorner pc[2];
      pix_pair(A, lg, T1, T2, pc);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int q = 2 * h + c;
        if (!ok[q]) continue;
        cs[t[q]] = pc[c];
        // corners on the leaf's boundary rows and columns: the seam cells'
        if (di[q] == 0 || di[q] == (uint32_t)(ni - 1) || dj[q] == 0 || dj[q] == (uint32_t)(nj - 1))
          edge[(j0 + (int64_t)dj[q] - A.grow0) * A.gnx1 + i0 + (int64_t)di[q]] = pc[c];
      }
    }
  }
  __shared__ int next_round;
  if (tid == 0) {
    atomicAdd(&I.stats[15], (double)ncorn);
    next_round = kFuseWarps;
  }
  __syncthreads();  // every corner in cs; the evaluation's staging becomes the IPM's
  // ---- IPM of the item's interior cells: 32 cells a round, each warp taking
  // the next round from a counter (cells near a star cost many times more)
  const int cw = it.w - 1, nc = cw > 0 && it.h > 1 ? cw * (it.h - 1) : 0;
  const int64_t crow0 = j0 + it.cj - A.grow0, ccol0 = i0 + it.ci;
  Ledger led;
  for (int rd = wp; rd * 32 < nc;) {
    const int idx = rd * 32 + lane;
    const bool has = idx < nc;
    int64_t cid = 0;
    PixCorner q4[4];
    if (has) {
      const int r = idx / cw, c = idx - r * cw;
      const int b = r * it.w + c;
      q4[0] = cs[b]; q4[1] = cs[b + 1]; q4[2] = cs[b + it.w + 1]; q4[3] = cs[b + it.w];
      cid = (crow0 + r) * I.nx + ccol0 + c;
    }
    ipm_round<true>(I, sm.m.c[wp], lane, has, cid, q4, led, sm.m.cut[wp]);
    __syncwarp();
    int nxt = 0;
    if (lane == 0) nxt = atomicAdd(&next_round, 1);
    rd = __shfl_sync(0xffffffffu, nxt, 0);
  }
  block_add_stats<kFuseWarps>(I.stats, led, I.wcell);
}

// Per active leaf: its work items and its seam cells (the chunk's cells on
// the leaf's last corner column or row).  jlast: the chunk's last cell row.
__global__ void k_fuse_count(const int64_t* __restrict__ rect, int64_t nl, int64_t nx, int64_t jlast,
                             int64_t* __restrict__ nitem, int64_t* __restrict__ nseam) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nl) return;
  const int64_t i0 = rect[4 * k], ni = rect[4 * k + 1], j0 = rect[4 * k + 2], nj = rect[4 * k + 3];
  if (ni <= 0 || nj <= 0) { nitem[k] = 0; nseam[k] = 0; return; }
  const int64_t sw = ni < kFuseSeg ? ni : kFuseSeg;
  const int64_t nseg = ni <= kFuseSeg ? 1 : (ni - 1 + kFuseSeg - 2) / (kFuseSeg - 1);
  const int64_t bh = min64(nj, max64(2, kFuseCorners / sw));
  const int64_t nband = nj <= bh ? 1 : (nj - 1 + bh - 2) / (bh - 1);
  nitem[k] = nseg * nband;
  const int64_t right = i0 + ni - 1 <= nx - 1 ? max64(0, min64(j0 + nj - 1, jlast) - j0 + 1) : 0;
  const int64_t top = j0 + nj - 1 <= jlast ? ni - 1 : 0;
  nseam[k] = right + top;
}

// One warp per active leaf: its items (segments x bands) and seam cell ids.
__global__ void k_fuse_fill(const int64_t* __restrict__ rect, int64_t nl, int64_t nx, int64_t jlast,
                            int64_t grow0, const int64_t* __restrict__ ioff,
                            const int64_t* __restrict__ soff, FuseItem* __restrict__ items,
                            int* __restrict__ seam) {
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nl) return;
  const int64_t i0 = rect[4 * k], ni = rect[4 * k + 1], j0 = rect[4 * k + 2], nj = rect[4 * k + 3];
  if (ni <= 0 || nj <= 0) return;
  const int64_t sw = ni < kFuseSeg ? ni : kFuseSeg;
  const int64_t nseg = ni <= kFuseSeg ? 1 : (ni - 1 + kFuseSeg - 2) / (kFuseSeg - 1);
  const int64_t bh = min64(nj, max64(2, kFuseCorners / sw));
  const int64_t nitems = ioff[k + 1] - ioff[k];
  for (int64_t e = lane; e < nitems; e += 32) {
    const int64_t b = e / nseg, sg = e - b * nseg;
    FuseItem it;
    it.leaf = (int)k;
    it.ci = (int)(sg * (kFuseSeg - 1));
    it.w = (int)min64(sw, ni - it.ci);
    it.cj = (int)(b * (bh - 1));
    it.h = (int)min64(bh, nj - it.cj);
    items[ioff[k] + e] = it;
  }
  const int64_t right = i0 + ni - 1 <= nx - 1 ? max64(0, min64(j0 + nj - 1, jlast) - j0 + 1) : 0;
  const int64_t ns = soff[k + 1] - soff[k];
  for (int64_t e = lane; e < ns; e += 32) {
    int64_t i, j;
    if (e < right) { i = i0 + ni - 1; j = j0 + e; }
    else { i = i0 + (e - right); j = j0 + nj - 1; }
    seam[soff[k] + e] = (int)((j - grow0) * nx + i);
  }
}

// ---- plan-time preparation ---------------------------------------------------
// per active leaf: centre, 1/r, r (the tree alone)
__global__ void k_prep_leaf_geo(const int* __restrict__ leaves, int64_t nl,
                                const int* __restrict__ level, const int* __restrict__ ix,
                                const int* __restrict__ iy, double lo_x, double lo_y, double size,
                                LeafPlan* __restrict__ out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nl) return;
  const int B = leaves[k];
  const double r = size / (double)(2ull << level[B]);
  LeafPlan lp;
  lp.cx = lo_x + (2.0 * ix[B] + 1.0) * r;
  lp.cy = lo_y + (2.0 * iy[B] + 1.0) * r;
  lp.K1 = 0.0; lp.K2 = 0.0;
  lp.ir = (float)(1.0 / r);
  lp.r = (float)r;
  out[k] = lp;
}

// per active leaf: the lens equation at the centre with the constant term of
// the local expansion, and the float32 local coefficients (the expansions)
__global__ void k_prep_leaf_exp(const int* __restrict__ leaves, int64_t nl, double a, double b,
                                int p, const double2* __restrict__ L, LeafPlan* __restrict__ out,
                                float2* __restrict__ fL) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nl) return;
  const int B = leaves[k];
  const double2* Lb = L + (int64_t)B * (p + 1);
  const double2 b0 = Lb[0];
  out[k].K1 = a * out[k].cx - b0.x;
  out[k].K2 = b * out[k].cy + b0.y;
  for (int l = 0; l <= p; ++l) fL[k * (int64_t)(p + 1) + l] = make_float2((float)Lb[l].x, (float)Lb[l].y);
}

// W boxes of at most this many stars are summed directly (P2P) instead of
// evaluated from their multipole (M2P): per ray, P2P costs ~8 float32
// operations per star against ~4(p+1) + 25 for one M2P.
inline int w_direct_max(int p) { return std::max(1, (p + 1) / 2); }

// Per active leaf: near boxes (U list + small W boxes), their stars, and the
// far W boxes.
__global__ void k_prep_counts(const int* __restrict__ leaves, int64_t nl, const int* __restrict__ aidx,
                              const int64_t* __restrict__ W_off,
                              const int* __restrict__ W_list, const int* __restrict__ count,
                              const int64_t* __restrict__ ustar_cnt, int wmax,
                              int64_t* __restrict__ scnt, int64_t* __restrict__ wcnt) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nl) return;
  const int a = aidx[leaves[k]];
  int64_t ns = ustar_cnt[a], nw = 0;
  for (int64_t e = W_off[a]; e < W_off[a + 1]; ++e) {
    const int c = count[W_list[e]];
    if (c <= wmax) ns += c; else ++nw;
  }
  scnt[k] = ns; wcnt[k] = nw;
}

__global__ void k_prep_lists(const int* __restrict__ leaves, int64_t nl, const int* __restrict__ aidx,
                             const LeafPlan* __restrict__ lp, const int64_t* __restrict__ U_off,
                             const int* __restrict__ U_list, const int64_t* __restrict__ W_off,
                             const int* __restrict__ W_list, const int* __restrict__ start,
                             const int* __restrict__ count, const int* __restrict__ level,
                             const int* __restrict__ ix, const int* __restrict__ iy, double lo_x,
                             double lo_y, double size, const double2* __restrict__ spos,
                             const double* __restrict__ smass, int wmax,
                             const int64_t* __restrict__ uoff, const int64_t* __restrict__ woff,
                             float4* __restrict__ ust, float* __restrict__ um,
                             int* __restrict__ wlist, float4* __restrict__ wgeo) {
  // One warp per active leaf.  Its candidate boxes (U leaves, then W boxes)
  // are taken 32 at a time, one per lane; the stars of the staged ones (U
  // leaves, W boxes of at most wmax stars) are then spread over the lanes,
  // so the float64 offsets run on full lanes and the loads in parallel.
  __shared__ int sh_incl[4][32], sh_st[4][32];
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wb = (threadIdx.x >> 5) & 3;
  if (k >= nl) return;
  const int a = aidx[leaves[k]];
  const double cx = lp[k].cx, cy = lp[k].cy;
  int64_t os = uoff[k], ow = woff[k];
  const int64_t u0 = U_off[a], nu = U_off[a + 1] - u0;
  const int64_t w0 = W_off[a], ntot = nu + (W_off[a + 1] - w0);
  for (int64_t e0 = 0; e0 < ntot; e0 += 32) {
    const int64_t e = e0 + lane;
    int C = -1, cnt = 0, st = 0;
    bool far = false;
    if (e < ntot) {
      C = e < nu ? U_list[u0 + e] : W_list[w0 + (e - nu)];
      const int c = count[C];
      if (e < nu || c <= wmax) { cnt = c; st = start[C]; } else { far = true; }
    }
    // far W boxes keep their order in wlist / wgeo
    const unsigned fm = __ballot_sync(0xffffffffu, far);
    if (far) {
      const int64_t slot = ow + __popc(fm & ((1u << lane) - 1u));
      const double r = size / (double)(2ull << level[C]);
      const double wx = lo_x + (2.0 * ix[C] + 1.0) * r, wy = lo_y + (2.0 * iy[C] + 1.0) * r;
      wlist[slot] = C;
      wgeo[slot] = make_float4((float)(wx - cx), (float)(wy - cy), (float)r, 0.f);
    }
    ow += __popc(fm);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    sh_incl[wb][lane] = incl;
    sh_st[wb][lane] = st;
    __syncwarp();
    for (int f0 = 0; f0 < total; f0 += 32) {
      const int f = f0 + lane;
      if (f < total) {
        int L = 0;  // first lane whose inclusive count exceeds f
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (sh_incl[wb][L + step - 1] <= f) L += step;
        const int j = sh_st[wb][L] + f - (L ? sh_incl[wb][L - 1] : 0);
        const double2 z = spos[j];
        const ff fx = ff_of(z.x - cx), fy = ff_of(z.y - cy);
        ust[os + f] = make_float4(fx.hi, fy.hi, fx.lo, fy.lo);
        um[os + f] = (float)smass[j];
      }
    }
    os += total;
  }
}

// float32 copies of the multipoles the float32 evaluation reads: those of the
// far W boxes (M2P), one thread per (list entry, coefficient); a box listed
// by several leaves is written with the same values by each
__global__ void k_to_f32(const int* __restrict__ wlist, int64_t nw, int P1,
                         const double2* __restrict__ M, float2* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nw * P1) return;
  const int64_t e = t / P1;
  const int64_t i = (int64_t)wlist[e] * P1 + (t - e * P1);
  out[i] = make_float2((float)M[i].x, (float)M[i].y);
}

// ---- per-call grid constants -------------------------------------------------
// Per-call leaf constants on the grid path.  parts & 1: the offset of the
// leaf's first grid ray from its centre (the tree alone); parts & 2: the
// pixel reference of the centre on the map path (needs the expansions).
__global__ void k_leaf_grid(int64_t nl, const LeafPlan* __restrict__ lp, const int64_t* __restrict__ rect,
                            double x0, double y0, double h, int64_t nx, int64_t ny, int parts,
                            double inv_du, double u_off, double inv_dv, double v_off,
                            LeafGrid* __restrict__ out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nl) return;
  const LeafPlan L = lp[k];
  if (parts & 1) {
    const double xi = __dadd_rn(x0, __dmul_rn((double)rect[4 * k], h));
    const double yj = __dadd_rn(y0, __dmul_rn((double)rect[4 * k + 2], h));
    out[k].bx = ff_of(xi - L.cx);
    out[k].by = ff_of(yj - L.cy);
    // the grid-unit origin: fixed by the leaf and the whole grid alone, so a
    // corner gets the same bits in every band; clamped into the grid, it lies
    // no farther from any of the leaf's rays than the leaf's rectangle spans
    const double gi = fmin(fmax(rint((L.cx - x0) / h), 0.0), (double)nx);
    const double gj = fmin(fmax(rint((L.cy - y0) / h), 0.0), (double)ny);
    out[k].rx = ff_of(__dadd_rn(x0, __dmul_rn(gi, h)) - L.cx);
    out[k].ry = ff_of(__dadd_rn(y0, __dmul_rn(gj, h)) - L.cy);
    out[k].ri = (int)(rect[4 * k] - (int64_t)gi);
    out[k].rj = (int)(rect[4 * k + 2] - (int64_t)gj);
  }
  if (parts & 2) {
    const double U1 = fma(L.K1, inv_du, u_off), V1 = fma(L.K2, inv_dv, v_off);
    const int far = !(fabs(U1) < 1073741824.0 && fabs(V1) < 1073741824.0);
    out[k].far = far;
    if (!far) {
      const double fu = floor(U1), fv = floor(V1);
      out[k].U1i = (int)fu; out[k].V1i = (int)fv;
      out[k].U1f = ff_of(U1 - fu); out[k].V1f = ff_of(V1 - fv);
    } else {
      out[k].U1i = 0; out[k].V1i = 0;
      out[k].U1f = ff{0.f, 0.f}; out[k].V1f = ff{0.f, 0.f};
    }
  }
}

E32Args base_args32(Plan& P) {
  E32Args A{};
  A.leaf = P.f_leaf; A.leaves = P.active_leaves; A.nleaf = P.n_active_leaves;
  A.aidx = P.box_aidx; A.count = P.box_count;
  A.woff = P.f_woff; A.wlist = P.f_wlist;
  A.fL = P.f_L; A.fM = P.f_M; A.ust = P.f_ust; A.um = P.f_um; A.uoff = P.f_uoff;
  A.wgeo = P.f_wgeo;
  A.p = P.p;
  A.a = 1.0 - P.kappa_s - P.gamma;
  A.b = 1.0 - P.kappa_s + P.gamma;
  A.af = ff_of(A.a);
  A.bf = ff_of(A.b);
  // a mass that float32 holds exactly (1, or any other with a short mantissa)
  A.unit_mass = P.equal_mass && (double)(float)P.mass0 == P.mass0;
  A.m0 = (float)P.mass0;
  return A;
}

template <bool GRID, bool PIX>
void launch32(E32Args& A, int64_t total, bool jac, cudaStream_t s) {
  if (total <= 0) return;
  if (total > (int64_t)INT32_MAX) fail(LENS_EINVAL, "too many ray tiles in one call");
  const unsigned g = (unsigned)total;
  if (jac) k_eval32<true, GRID, PIX><<<g, kT, 0, s>>>(A);
  else if (A.unit_mass) k_eval32<false, GRID, PIX, true><<<g, kT, 0, s>>>(A);
  else k_eval32<false, GRID, PIX><<<g, kT, 0, s>>>(A);
  LENS_LAUNCHED("k_eval32");
}

}  // namespace

void eval32_alloc(Plan& P) {
  const int64_t nl = P.n_active_leaves;
  const int P1 = P.p + 1;
  P.f_leaf = P.dalloc_n<LeafPlan>(nl);
  P.f_L = P.dalloc_n<float2>((size_t)nl * P1);
  P.f_M = P.dalloc_n<float2>((size_t)P.nb * P1);
  P.f_uoff = P.dalloc_n<int64_t>(nl + 1);
  P.f_woff = P.dalloc_n<int64_t>(nl + 1);
  P.f_ncnt = P.dalloc_n<int64_t>(nl + 1);
  P.f_wcnt = P.dalloc_n<int64_t>(nl + 1);
}

void eval32_prepare_tree(Plan& P, cudaStream_t s) {
  const int64_t nl = P.n_active_leaves;
  if (nl == 0) return;
  const int wmax = w_direct_max(P.p);
  k_prep_leaf_geo<<<grid_for(nl, 128), 128, 0, s>>>(P.active_leaves, nl, P.box_level, P.box_ix,
                                                    P.box_iy, P.root_lo[0], P.root_lo[1],
                                                    P.root_size, P.f_leaf);
  LENS_LAUNCHED("k_prep_leaf_geo");
  LENS_CUDA(cudaMemsetAsync(P.f_ncnt, 0, sizeof(int64_t) * (nl + 1), s));
  LENS_CUDA(cudaMemsetAsync(P.f_wcnt, 0, sizeof(int64_t) * (nl + 1), s));
  k_prep_counts<<<grid_for(nl, 128), 128, 0, s>>>(P.active_leaves, nl, P.box_aidx, P.W_off,
                                                  P.W_list, P.box_count, P.ustar_cnt, wmax,
                                                  P.f_ncnt, P.f_wcnt);
  LENS_LAUNCHED("k_prep_counts");
  exclusive_scan_i64(P.f_ncnt, P.f_uoff, nl + 1, P.da, s);
  exclusive_scan_i64(P.f_wcnt, P.f_woff, nl + 1, P.da, s);
  int64_t tot[2] = {0, 0};
  const int64_t* addr[2] = {P.f_uoff + nl, P.f_woff + nl};
  read_i64(addr, 2, tot, P.da, s);
  P.f_ust = P.dalloc_n<float4>(tot[0]);
  P.f_um = P.dalloc_n<float>(tot[0]);
  P.f_wlist = P.dalloc_n<int>(tot[1]);
  P.f_nw = tot[1];
  P.f_wgeo = P.dalloc_n<float4>(tot[1]);
  k_prep_lists<<<grid_for(nl * 32, 128), 128, 0, s>>>(
      P.active_leaves, nl, P.box_aidx, P.f_leaf, P.U_off, P.U_list, P.W_off, P.W_list,
      P.box_start, P.box_count, P.box_level, P.box_ix, P.box_iy, P.root_lo[0], P.root_lo[1],
      P.root_size, P.spos, P.smass, wmax, P.f_uoff, P.f_woff, P.f_ust, P.f_um, P.f_wlist,
      P.f_wgeo);
  LENS_LAUNCHED("k_prep_lists");
}

void eval32_prepare_expansions(Plan& P, cudaStream_t s) {
  const int64_t nl = P.n_active_leaves;
  const int P1 = P.p + 1;
  const double a = 1.0 - P.kappa_s - P.gamma, b = 1.0 - P.kappa_s + P.gamma;
  if (nl > 0) {
    k_prep_leaf_exp<<<grid_for(nl, 128), 128, 0, s>>>(P.active_leaves, nl, a, b, P.p, P.L,
                                                      P.f_leaf, P.f_L);
    LENS_LAUNCHED("k_prep_leaf_exp");
  }
  if (P.f_nw > 0) {
    k_to_f32<<<grid_for(P.f_nw * P1, 256), 256, 0, s>>>(P.f_wlist, P.f_nw, P1, P.M, P.f_M);
    LENS_LAUNCHED("k_to_f32");
  }
}

void eval32_grid(Plan& P, const GridRows& g, const int64_t* rect, const int2* tile_leaf,
                 int64_t total, double* y, double* jac, PixCorner* pix, const IpmParams* ip,
                 cudaStream_t s) {
  const int64_t nl = P.n_active_leaves;
  Scratch lg(&P.da, sizeof(LeafGrid) * (nl + 1));
  const bool px = pix != nullptr;
  auto leaf_grid = [&](int parts) {
    k_leaf_grid<<<grid_for(nl, 128), 128, 0, s>>>(
        nl, P.f_leaf, rect, g.x0, g.y0, g.h, g.nx, g.ny, parts, px ? ip->inv_du : 0.0,
        px ? -ip->u0 * ip->inv_du : 0.0, px ? ip->inv_dv : 0.0, px ? -ip->v0 * ip->inv_dv : 0.0,
        lg.as<LeafGrid>());
    LENS_LAUNCHED("k_leaf_grid");
  };
  E32Args A = base_args32(P);
  A.tile_leaf = tile_leaf;
  A.rect = rect;
  A.lgrid = lg.as<LeafGrid>();
  A.hf = ff_of(g.h);
  A.ihf = ff_of(1.0 / g.h);
  A.gnx1 = g.nx + 1;
  A.grow0 = g.row0;
  A.y = y; A.jac = jac; A.pix = pix;
  if (px) { A.iduf = ff_of(ip->inv_du); A.idvf = ff_of(ip->inv_dv); }
  wait_expansions(P, s);
  leaf_grid(px ? 3 : 1);
  // kernel time only: the events follow the wait for the plan's expansions
  std::pair<cudaEvent_t, cudaEvent_t> e;
  if (P.timing) e = event_pair_begin(s);
  if (px) launch32<true, true>(A, total, false, s);
  else launch32<true, false>(A, total, jac != nullptr, s);
  if (P.timing) {
    event_pair_end(e, s);
    P.ev_eval.push_back(e);
  }
}

Scratch eval32_fused(Plan& P, const GridRows& g, const int64_t* rect, PixCorner* edge,
                     const IpmParams& ip, float* map32, float* rowdiff, double* stats_dev, int* rq,
                     int* rqcount, int64_t& nseam, cudaStream_t s) {
  const int64_t nl = P.n_active_leaves;
  const int64_t jlast = g.row0 + g.nrows - 2;  // the chunk's last cell row
  Scratch cnt(&P.da, sizeof(int64_t) * (nl + 1)), scnt(&P.da, sizeof(int64_t) * (nl + 1));
  Scratch ioff(&P.da, sizeof(int64_t) * (nl + 1)), soff(&P.da, sizeof(int64_t) * (nl + 1));
  LENS_CUDA(cudaMemsetAsync(cnt.as<int64_t>() + nl, 0, sizeof(int64_t), s));
  LENS_CUDA(cudaMemsetAsync(scnt.as<int64_t>() + nl, 0, sizeof(int64_t), s));
  k_fuse_count<<<grid_for(nl, 128), 128, 0, s>>>(rect, nl, g.nx, jlast, cnt.as<int64_t>(),
                                                 scnt.as<int64_t>());
  LENS_LAUNCHED("k_fuse_count");
  exclusive_scan_i64(cnt.as<int64_t>(), ioff.as<int64_t>(), nl + 1, P.da, s);
  exclusive_scan_i64(scnt.as<int64_t>(), soff.as<int64_t>(), nl + 1, P.da, s);
  int64_t tot[2] = {0, 0};
  const int64_t* addr[2] = {ioff.as<int64_t>() + nl, soff.as<int64_t>() + nl};
  read_i64(addr, 2, tot, P.da, s);
  const int64_t nitems = tot[0];
  nseam = tot[1];
  if (nitems > (int64_t)INT32_MAX) fail(LENS_EINVAL, "too many work items in one chunk");
  Scratch items(&P.da, sizeof(FuseItem) * (size_t)std::max<int64_t>(nitems, 1));
  Scratch seam(&P.da, sizeof(int) * (size_t)std::max<int64_t>(nseam, 1));
  k_fuse_fill<<<grid_for(nl * 32, 128), 128, 0, s>>>(rect, nl, g.nx, jlast, g.row0,
                                                    ioff.as<int64_t>(), soff.as<int64_t>(),
                                                    items.as<FuseItem>(), seam.as<int>());
  LENS_LAUNCHED("k_fuse_fill");
  Scratch lg(&P.da, sizeof(LeafGrid) * (nl + 1));
  E32Args A = base_args32(P);
  A.rect = rect;
  A.lgrid = lg.as<LeafGrid>();
  A.hf = ff_of(g.h);
  A.ihf = ff_of(1.0 / g.h);
  A.gnx1 = g.nx + 1;
  A.grow0 = g.row0;
  A.iduf = ff_of(ip.inv_du);
  A.idvf = ff_of(ip.inv_dv);
  IpmArgs I{};
  I.nx = g.nx; I.map = map32; I.D = rowdiff; I.ldd = (int64_t)ip.npx + 1; I.stats = stats_dev;
  I.ip = ip; I.wcell = 1.f; I.rq = rq; I.rqcount = rqcount;
  ipm_prepare(I);
  wait_expansions(P, s);
  k_leaf_grid<<<grid_for(nl, 128), 128, 0, s>>>(nl, P.f_leaf, rect, g.x0, g.y0, g.h, g.nx, g.ny, 3,
                                                ip.inv_du,
                                                -ip.u0 * ip.inv_du, ip.inv_dv, -ip.v0 * ip.inv_dv,
                                                lg.as<LeafGrid>());
  LENS_LAUNCHED("k_leaf_grid");
  std::pair<cudaEvent_t, cudaEvent_t> e;
  if (P.timing) e = event_pair_begin(s);
  if (nitems > 0) {
    if (A.unit_mass) k_eval32_map<true><<<(unsigned)nitems, kT, 0, s>>>(A, I, items.as<FuseItem>(), edge);
    else k_eval32_map<false><<<(unsigned)nitems, kT, 0, s>>>(A, I, items.as<FuseItem>(), edge);
    LENS_LAUNCHED("k_eval32_map");
  }
  if (P.timing) {
    event_pair_end(e, s);
    P.ev_fused.push_back(e);
  }
  return seam;
}

void eval32_rays(Plan& P, const double* rays, const int64_t* off, const int* perm,
                 const int2* tile_leaf, int64_t total, double* y, double* jac, cudaStream_t s) {
  wait_expansions(P, s);
  E32Args A = base_args32(P);
  A.tile_leaf = tile_leaf;
  A.rays = rays; A.ray_off = off; A.perm = perm;
  A.y = y; A.jac = jac;
  launch32<false, false>(A, total, jac != nullptr, s);
}

}  // namespace lens
