// adjoint.cu -- transposed FMM: gradient of a loss through Eq. 1 with respect
// to the star positions, masses, kappa_s and gamma (not in the paper; the
// forward operators are those of Appendix A, run backwards on the same tree).
//
// With f(z) = sum_j m_j/(z - z_j), alpha = conj(f) and g = dL/dy at every ray,
// dL/dalpha = -g, so dL = Re sum_r c_r df_r with the ray charge
// c_r = -(g1 + i g2).  Every forward step is complex-linear in its input, so
// its adjoint is its plain transpose (dL = Re sum_l Lhat_l dB_l):
//   L2P^T  Lhat_B,l   += sum_{r in B} c_r w_r^l           (w = (z_r - c_B)/r_B)
//   M2P^T  Mhat_C,k   += sum_{r} c_r q_r^k / (z_r - c_C)   (q = r_C/(z_r - c_C), W lists)
//   P2P^T  Phi_j      += c_r/(z_r - z_j),  Psi_j += c_r m_j/(z_r - z_j)^2   (U lists)
//   L2L^T  Lhat_P,l   += sum_{j<=l} S_q[j][l] Lhat_C,j      (children -> parent)
//   M2L^T  Mhat_C,k   += u^k sum_l C(k+l,k) (-1)^l u^(l+1) Lhat_B,l / r   (V lists)
//   P2L^T  Phi_j += sum_l Lhat_B,l (-q^l/(z_j-c)),  Psi_j += sum_l Lhat_B,l m_j (l+1) q^l/(z_j-c)^2  (X)
//   M2M^T  Mhat_C,k   += sum_{l>=k} T_q[l][k] Mhat_P,l     (parent -> children)
//   P2M^T  Phi_j += sum_k Mhat_k w_j^k,  Psi_j += m_j sum_k k Mhat_k w_j^(k-1)/r  (leaves)
// where Phi_j, Psi_j give dL/dm_j = Re Phi_j and dL/dz_j = Psi_j, i.e.
// dL/dx_j = Re Psi_j, dL/dy_j = -Im Psi_j.  The smooth field adds
// dL/dkappa_s = -sum_r (g1 x1 + g2 x2), dL/dgamma = sum_r (-g1 x1 + g2 x2).
// For float64 plans everything here is float64; float32-bulk plans run the
// per-ray and per-pair operators in float32 (below).  Deterministic up to the
// order of atomic adds.
#include <cmath>

#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kAdjTile = 128;  // rays per tile
constexpr int kAdjU = 64;      // U-list leaves staged at a time by k_adj_p2p32

__device__ __forceinline__ void atomic_add2(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

struct AdjArgs {
  const double* rays; const double* gy;
  const int* perm; const int64_t* ray_off; const int64_t* tile_off; int64_t nleaf;
  const int* leaves; const int* aidx; const int* level; const int* ix; const int* iy;
  const int* start; const int* count; const int* child; const int* parent;
  const int64_t* U_off; const int* U_list; const int64_t* W_off; const int* W_list;
  const int64_t* V_off; const int* V_list; const int64_t* X_off; const int* X_list;
  const double2* spos; const double* smass;
  FmmTables tab;
  double lo_x, lo_y, size;
  int p;
  double2* Lh; double2* Mh;   // adjoints of L (by box) and M (by box)
  double2* Phi; double2* Psi; // per sorted star
  double* gkg;                // [2]
};

__device__ __forceinline__ int64_t leaf_of_tile(const int64_t* toff, int64_t nleaf, int64_t b) {
  int64_t lo = 0, hi = nleaf;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (toff[mid] <= b) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double box_r(const AdjArgs& A, int b) {
  return A.size / (double)(2ull << A.level[b]);
}
__device__ __forceinline__ double2 box_c(const AdjArgs& A, int b, double r) {
  return make_double2(A.lo_x + (2.0 * A.ix[b] + 1.0) * r, A.lo_y + (2.0 * A.iy[b] + 1.0) * r);
}

// One warp per (leaf, tile): L2P^T moments of the tile's rays and M2P^T for
// every W entry, accumulated per lane in shared memory, reduced, and added
// atomically (tiles of one leaf share Lhat_B).
__global__ void __launch_bounds__(32) k_adj_leaf_moments(AdjArgs A) {
  extern __shared__ double2 acc[];  // [(p+1)][32]
  const int lane = threadIdx.x;
  const int64_t k = leaf_of_tile(A.tile_off, A.nleaf, blockIdx.x);
  const int B = A.leaves[k];
  const int a = A.aidx[B];
  const int64_t tile = (int64_t)blockIdx.x - A.tile_off[k];
  const int64_t n = A.ray_off[k + 1] - A.ray_off[k];
  const int64_t r0 = tile * kAdjTile;
  const int64_t r1 = min64(n, r0 + kAdjTile);
  const int p = A.p;
  const double rB = box_r(A, B);
  const double2 cB = box_c(A, B, rB);
  const double irB = 1.0 / rB;
  // pass 0: L2P^T; pass e >= 1: M2P^T of W entry e-1
  const int64_t nW = A.W_off[a + 1] - A.W_off[a];
  for (int64_t pass = 0; pass <= nW; ++pass) {
    for (int l = 0; l <= p; ++l) acc[l * 32 + lane] = make_double2(0.0, 0.0);
    int C = -1;
    double rC = 0;
    double2 cC = make_double2(0, 0);
    if (pass > 0) {
      C = A.W_list[A.W_off[a] + pass - 1];
      rC = box_r(A, C);
      cC = box_c(A, C, rC);
    }
    for (int64_t t = r0 + lane; t < r1; t += 32) {
      const int64_t ridx = A.perm[A.ray_off[k] + t];
      const double2 z = make_double2(A.rays[2 * ridx], A.rays[2 * ridx + 1]);
      const double2 c = make_double2(-A.gy[2 * ridx], -A.gy[2 * ridx + 1]);
      double2 pw, w;
      if (pass == 0) {
        w = make_double2((z.x - cB.x) * irB, (z.y - cB.y) * irB);
        pw = c;
      } else {
        const double2 inv = cinv(make_double2(z.x - cC.x, z.y - cC.y));
        w = make_double2(inv.x * rC, inv.y * rC);
        pw = cmul(c, inv);
      }
      for (int l = 0; l <= p; ++l) {
        acc[l * 32 + lane] = acc[l * 32 + lane] + pw;
        pw = cmul(pw, w);
      }
    }
    __syncwarp();
    double2* dst = pass == 0 ? A.Lh + (int64_t)B * (p + 1) : A.Mh + (int64_t)C * (p + 1);
    for (int l = 0; l <= p; ++l) {
      double2 v = acc[l * 32 + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      }
      if (lane == 0 && (v.x != 0.0 || v.y != 0.0)) atomic_add2(dst + l, v);
    }
    __syncwarp();
  }
}

// P2P^T: threads over the U-list stars of the tile's leaf, rays of the tile
// staged in shared memory.
__global__ void __launch_bounds__(128) k_adj_p2p(AdjArgs A) {
  __shared__ double2 sz[kAdjTile], sc[kAdjTile];
  const int64_t k = leaf_of_tile(A.tile_off, A.nleaf, blockIdx.x);
  const int B = A.leaves[k];
  const int a = A.aidx[B];
  const int64_t tile = (int64_t)blockIdx.x - A.tile_off[k];
  const int64_t n = A.ray_off[k + 1] - A.ray_off[k];
  const int64_t r0 = tile * kAdjTile;
  const int nr = (int)min64(kAdjTile, n - r0);
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    const int64_t ridx = A.perm[A.ray_off[k] + r0 + t];
    sz[t] = make_double2(A.rays[2 * ridx], A.rays[2 * ridx + 1]);
    sc[t] = make_double2(-A.gy[2 * ridx], -A.gy[2 * ridx + 1]);
  }
  __syncthreads();
  // flatten the U-list stars: walk entries, threads take stars in turn
  int64_t base = 0;
  for (int64_t e = A.U_off[a]; e < A.U_off[a + 1]; ++e) {
    const int C = A.U_list[e];
    const int s0 = A.start[C], ns = A.count[C];
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
      const int sj = s0 + j;
      const double2 zj = A.spos[sj];
      const double mj = A.smass[sj];
      double2 F = make_double2(0, 0), G = make_double2(0, 0);
      for (int t = 0; t < nr; ++t) {
        const double2 d = make_double2(sz[t].x - zj.x, sz[t].y - zj.y);
        if (d.x == 0.0 && d.y == 0.0) continue;  // self-interaction skipped
        const double2 inv = cinv(d);
        const double2 ci = cmul(sc[t], inv);
        F = F + ci;
        G = G + cmul(ci, inv);
      }
      atomic_add2(A.Phi + sj, F);
      atomic_add2(A.Psi + sj, make_double2(mj * G.x, mj * G.y));
    }
    base += ns;
  }
}

// ---- float32 bulk (plans of precision LENS_FP32_BULK) ------------------------
// The per-ray and per-pair parts of the adjoint in float32, as the forward
// pass evaluates them: P2P^T on float-float offsets from the leaf centre
// (each pair's difference exact to float32 rounding however close a ray is
// to a star), partial sums compensated; L2P^T / M2P^T moments with the
// scaled offsets w rounded once to float32 (|w| <= ~1.5: no cancellation),
// summed per lane in float32 and across lanes in float64.  The transposed
// translations (L2L^T, M2L^T, P2L^T, M2M^T, P2M^T) stay float64.

// P2P^T: block per (leaf, tile of rays), threads over the U-list stars; the
// tile's rays staged as float-float offsets from the leaf centre with their
// float32 charges.
__global__ void __launch_bounds__(128) k_adj_p2p32(AdjArgs A) {
  __shared__ float4 sz[kAdjTile];  // x_hi, y_hi, x_lo, y_lo
  __shared__ float2 sc[kAdjTile];
  const int64_t k = leaf_of_tile(A.tile_off, A.nleaf, blockIdx.x);
  const int B = A.leaves[k];
  const int a = A.aidx[B];
  const int64_t tile = (int64_t)blockIdx.x - A.tile_off[k];
  const int64_t n = A.ray_off[k + 1] - A.ray_off[k];
  const int64_t r0 = tile * kAdjTile;
  const int nr = (int)min64(kAdjTile, n - r0);
  const double rB = box_r(A, B);
  const double2 cB = box_c(A, B, rB);
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    const int64_t ridx = A.perm[A.ray_off[k] + r0 + t];
    const ff ox = ff_of(A.rays[2 * ridx] - cB.x), oy = ff_of(A.rays[2 * ridx + 1] - cB.y);
    sz[t] = make_float4(ox.hi, oy.hi, ox.lo, oy.lo);
    sc[t] = make_float2((float)-A.gy[2 * ridx], (float)-A.gy[2 * ridx + 1]);
  }
  // the stars of the U-list leaves, flattened over the block's threads (a
  // leaf's own count is often below the block size): up to kAdjU leaves at a
  // time, their first star and inclusive star counts in shared memory
  __shared__ int su_start[kAdjU], su_incl[kAdjU];
  const int64_t u0 = A.U_off[a], nu = A.U_off[a + 1] - u0;
  for (int64_t ub = 0; ub < nu; ub += kAdjU) {
    const int nub = (int)min64(kAdjU, nu - ub);
    __syncthreads();  // the previous group's readers are done (and the rays staged)
    if (threadIdx.x < nub) {
      const int C = A.U_list[u0 + ub + threadIdx.x];
      su_start[threadIdx.x] = A.start[C];
      su_incl[threadIdx.x] = A.count[C];
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 1; i < nub; ++i) su_incl[i] += su_incl[i - 1];
    __syncthreads();
    const int tot = su_incl[nub - 1];
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
      // the group's leaf holding flattened star q: the first with su_incl > q
      int lo = 0, hi = nub - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (su_incl[mid] > q) hi = mid; else lo = mid + 1;
      }
      const int sj = su_start[lo] + q - (lo ? su_incl[lo - 1] : 0);
      const double2 zj = A.spos[sj];
      const ff sx = ff_of(zj.x - cB.x), sy = ff_of(zj.y - cB.y);
      fcomp F1{0.f, 0.f}, F2{0.f, 0.f}, G1{0.f, 0.f}, G2{0.f, 0.f};
      for (int t = 0; t < nr; ++t) {
        const float4 z = sz[t];
        const float2 c = sc[t];
        // d = z_r - z_j; 1/d = conj(d) / |d|^2 (a star exactly at the ray adds
        // nothing: d = 0 makes both terms 0 under the floor on |d|^2)
        const float d1 = (z.x - sx.hi) + (z.z - sx.lo), d2 = (z.y - sy.hi) + (z.w - sy.lo);
        const float w = frcp_fast(fmaf(d1, d1, fmaf(d2, d2, 1e-30f)));
        const float i1 = d1 * w, i2 = -d2 * w;
        const float c1 = c.x * i1 - c.y * i2, c2 = c.x * i2 + c.y * i1;  // c / d
        F1.add(c1); F2.add(c2);
        G1.add(c1 * i1 - c2 * i2); G2.add(c1 * i2 + c2 * i1);             // c / d^2
      }
      const double mj = A.smass[sj];
      atomic_add2(A.Phi + sj, make_double2(F1.value(), F2.value()));
      atomic_add2(A.Psi + sj, make_double2(mj * G1.value(), mj * G2.value()));
    }
  }
}

// L2P^T and M2P^T moments in float32: one warp per (leaf, tile), as
// k_adj_leaf_moments.
__global__ void __launch_bounds__(32) k_adj_leaf_moments32(AdjArgs A) {
  extern __shared__ float2 acc32[];  // [(p+1)][33]: lane partials, padded
  const int lane = threadIdx.x;
  const int64_t k = leaf_of_tile(A.tile_off, A.nleaf, blockIdx.x);
  const int B = A.leaves[k];
  const int a = A.aidx[B];
  const int64_t tile = (int64_t)blockIdx.x - A.tile_off[k];
  const int64_t n = A.ray_off[k + 1] - A.ray_off[k];
  const int64_t r0 = tile * kAdjTile;
  const int64_t r1 = min64(n, r0 + kAdjTile);
  const int p = A.p;
  const double rB = box_r(A, B);
  const double2 cB = box_c(A, B, rB);
  const double irB = 1.0 / rB;
  const int64_t nW = A.W_off[a + 1] - A.W_off[a];
  for (int64_t pass = 0; pass <= nW; ++pass) {
    for (int l = 0; l <= p; ++l) acc32[l * 33 + lane] = make_float2(0.f, 0.f);
    int C = -1;
    double rC = 0;
    double2 cC = make_double2(0, 0);
    if (pass > 0) {
      C = A.W_list[A.W_off[a] + pass - 1];
      rC = box_r(A, C);
      cC = box_c(A, C, rC);
    }
    for (int64_t t = r0 + lane; t < r1; t += 32) {
      const int64_t ridx = A.perm[A.ray_off[k] + t];
      const float2 c = make_float2((float)-A.gy[2 * ridx], (float)-A.gy[2 * ridx + 1]);
      float2 pw, w;
      if (pass == 0) {
        w = make_float2((float)((A.rays[2 * ridx] - cB.x) * irB),
                        (float)((A.rays[2 * ridx + 1] - cB.y) * irB));
        pw = c;
      } else {
        const float2 inv = cinv(make_float2((float)(A.rays[2 * ridx] - cC.x),
                                            (float)(A.rays[2 * ridx + 1] - cC.y)));
        w = make_float2(inv.x * (float)rC, inv.y * (float)rC);
        pw = cmul(c, inv);
      }
      for (int l = 0; l <= p; ++l) {
        acc32[l * 33 + lane] = acc32[l * 33 + lane] + pw;
        pw = cmul(pw, w);
      }
    }
    __syncwarp();
    double2* dst = pass == 0 ? A.Lh + (int64_t)B * (p + 1) : A.Mh + (int64_t)C * (p + 1);
    // lane l sums order l's 32 lane partials in float64 (a float64 shuffle
    // tree would run the adds on every lane of every order)
    for (int l = lane; l <= p; l += 32) {
      double vx = 0.0, vy = 0.0;
      for (int q = 0; q < 32; ++q) {
        const float2 vf = acc32[l * 33 + q];
        vx += vf.x;
        vy += vf.y;
      }
      if (vx != 0.0 || vy != 0.0) atomic_add2(dst + l, make_double2(vx, vy));
    }
    __syncwarp();
  }
}

// L2L^T for one level: warp per active child box, adds into its parent.
__global__ void __launch_bounds__(128) k_adj_l2l(AdjArgs A, const int* active, int64_t a0, int64_t a1) {
  const int lane = threadIdx.x & 31;
  const int64_t ai = a0 + (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  if (ai >= a1) return;
  const int C = active[ai];
  const int P = A.parent[C];
  const int q = C - A.child[P];
  const int P1 = A.p + 1;
  const double2* S = A.tab.l2l + (int64_t)q * P1 * P1;
  const double2* Lc = A.Lh + (int64_t)C * P1;
  for (int l = lane; l <= A.p; l += 32) {
    double2 v = make_double2(0, 0);
    for (int j = 0; j <= l; ++j) v = cfma(S[j * P1 + l], Lc[j], v);
    if (v.x != 0.0 || v.y != 0.0) atomic_add2(A.Lh + (int64_t)P * P1 + l, v);
  }
}

// M2L^T (V) and P2L^T (X): warp per active box.
__global__ void __launch_bounds__(128) k_adj_m2l(AdjArgs A, const int* active, int64_t na) {
  __shared__ double2 sbuf[4][kMaxOrder + 2];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t ai = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  if (ai >= na) return;
  const int B = active[ai];
  const int p = A.p, P1 = p + 1;
  const double r = box_r(A, B);
  const double ir = 1.0 / r;
  const double2 cB = box_c(A, B, r);
  const double2* Lb = A.Lh + (int64_t)B * P1;
  double2* buf = sbuf[wib];
  for (int64_t e = A.V_off[ai]; e < A.V_off[ai + 1]; ++e) {
    const int C = A.V_list[e];
    const int dx = A.ix[C] - A.ix[B], dy = A.iy[C] - A.iy[B];
    const double2* up = A.tab.upow + (int64_t)((dy + 3) * 7 + (dx + 3)) * (p + 2);
    for (int l = lane; l <= p; l += 32) {
      double2 v = cmul(Lb[l], up[l + 1]);
      if (l & 1) v = make_double2(-v.x, -v.y);
      buf[l] = make_double2(v.x * ir, v.y * ir);
    }
    __syncwarp();
    for (int kk = lane; kk <= p; kk += 32) {
      double sx = 0, sy = 0;
      for (int l = 0; l <= p; ++l) {
        const double c = A.tab.binom[(int64_t)(kk + l) * A.tab.ldb + l];  // C(k+l, l)
        sx = fma(c, buf[l].x, sx);
        sy = fma(c, buf[l].y, sy);
      }
      const double2 v = cmul(up[kk], make_double2(sx, sy));
      if (v.x != 0.0 || v.y != 0.0) atomic_add2(A.Mh + (int64_t)C * P1 + kk, v);
    }
    __syncwarp();
  }
  for (int64_t e = A.X_off[ai]; e < A.X_off[ai + 1]; ++e) {
    const int C = A.X_list[e];
    for (int j = A.start[C]; j < A.start[C] + A.count[C]; ++j) {
      const double2 z = A.spos[j];
      const double m = A.smass[j];
      const double2 inv = cinv(make_double2(z.x - cB.x, z.y - cB.y));
      const double2 q = make_double2(inv.x * r, inv.y * r);
      double2 F = make_double2(0, 0), G = make_double2(0, 0);
      for (int l = lane; l <= p; l += 32) {
        double2 pw = make_double2(1.0, 0.0), bse = q;
        for (int e2 = l; e2 > 0; e2 >>= 1) {
          if (e2 & 1) pw = cmul(pw, bse);
          bse = cmul(bse, bse);
        }
        const double2 t = cmul(Lb[l], pw);
        F = F + t;
        G = G + make_double2((l + 1) * t.x, (l + 1) * t.y);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        F.x += __shfl_xor_sync(0xffffffffu, F.x, o); F.y += __shfl_xor_sync(0xffffffffu, F.y, o);
        G.x += __shfl_xor_sync(0xffffffffu, G.x, o); G.y += __shfl_xor_sync(0xffffffffu, G.y, o);
      }
      if (lane == 0) {
        const double2 Fj = cmul(F, inv);                 // sum Lhat q^l / (z - c)
        const double2 Gj = cmul(G, cmul(inv, inv));      // sum Lhat (l+1) q^l / (z - c)^2
        atomic_add2(A.Phi + j, make_double2(-Fj.x, -Fj.y));
        atomic_add2(A.Psi + j, make_double2(m * Gj.x, m * Gj.y));
      }
    }
  }
}

// M2M^T for one level: warp per box of the level, from its parent's Mhat.
__global__ void __launch_bounds__(128) k_adj_m2m(AdjArgs A, int64_t b0, int64_t b1) {
  const int lane = threadIdx.x & 31;
  const int64_t C = b0 + (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  if (C >= b1) return;
  if (A.count[C] == 0) return;
  const int P = A.parent[C];
  const int q = (int)C - A.child[P];
  const int P1 = A.p + 1;
  const double2* T = A.tab.m2m + (int64_t)q * P1 * P1;
  const double2* Mp = A.Mh + (int64_t)P * P1;
  for (int kk = lane; kk <= A.p; kk += 32) {
    double2 v = A.Mh[C * P1 + kk];
    for (int l = kk; l <= A.p; ++l) v = cfma(T[l * P1 + kk], Mp[l], v);
    A.Mh[C * P1 + kk] = v;
  }
}

// P2M^T at the stars of every leaf (thread per leaf).
__global__ void k_adj_p2m(AdjArgs A, int64_t nb) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nb || A.child[b] >= 0 || A.count[b] == 0) return;
  const int p = A.p, P1 = p + 1;
  const double r = box_r(A, (int)b);
  const double2 c = box_c(A, (int)b, r);
  const double ir = 1.0 / r;
  const double2* Mb = A.Mh + b * P1;
  for (int j = A.start[b]; j < A.start[b] + A.count[b]; ++j) {
    const double2 z = A.spos[j];
    const double m = A.smass[j];
    const double2 w = make_double2((z.x - c.x) * ir, (z.y - c.y) * ir);
    double2 F = Mb[p], G = make_double2(p * Mb[p].x, p * Mb[p].y);
    for (int kk = p - 1; kk >= 0; --kk) {
      F = cfma(F, w, Mb[kk]);
      if (kk >= 1) G = cfma(G, w, make_double2(kk * Mb[kk].x, kk * Mb[kk].y));
    }
    // G = sum_{k>=1} k Mhat_k w^(k-1)
    A.Phi[j] = A.Phi[j] + F;
    A.Psi[j] = A.Psi[j] + make_double2(m * G.x * ir, m * G.y * ir);
  }
}

__global__ void k_adj_kg(const double* rays, const double* gy, int64_t m, double* gkg) {
  __shared__ double sh[2][256];
  double sk = 0, sg = 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double x1 = rays[2 * r], x2 = rays[2 * r + 1], g1 = gy[2 * r], g2 = gy[2 * r + 1];
    sk -= g1 * x1 + g2 * x2;
    sg += -g1 * x1 + g2 * x2;
  }
  sh[0][threadIdx.x] = sk; sh[1][threadIdx.x] = sg;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) { sh[0][threadIdx.x] += sh[0][threadIdx.x + o]; sh[1][threadIdx.x] += sh[1][threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { atomicAdd(&gkg[0], sh[0][0]); atomicAdd(&gkg[1], sh[1][0]); }
}

__global__ void k_adj_out(const double2* Phi, const double2* Psi, const uint32_t* sidx, int64_t n,
                          double* gxy, double* gm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j = sidx[i];
  if (gm) gm[j] = Phi[i].x;
  if (gxy) { gxy[2 * j] = Psi[i].x; gxy[2 * j + 1] = -Psi[i].y; }
}

}  // namespace

void adjoint(Plan& P, const double* rays, int64_t m, const double* gy, double* gxy, double* gm,
             double* gkg, cudaStream_t s) {
  const int P1 = P.p + 1;
  wait_tree(P, s);  // the transposed operators need the tree, not the expansions
  if (gkg) LENS_CUDA(cudaMemsetAsync(gkg, 0, sizeof(double) * 2, s));
  if (m == 0) {
    if (gm) LENS_CUDA(cudaMemsetAsync(gm, 0, sizeof(double) * P.n, s));
    if (gxy) LENS_CUDA(cudaMemsetAsync(gxy, 0, sizeof(double) * 2 * P.n, s));
    return;
  }
  RayBuckets RB;
  bucket_rays(P, rays, m, kAdjTile, RB, s);
  Scratch Lh(&P.da, sizeof(double2) * (size_t)P.nb * P1);
  Scratch Mh(&P.da, sizeof(double2) * (size_t)P.nb * P1);
  Scratch Phi(&P.da, sizeof(double2) * (size_t)P.n), Psi(&P.da, sizeof(double2) * (size_t)P.n);
  LENS_CUDA(cudaMemsetAsync(Lh.p, 0, Lh.bytes, s));
  LENS_CUDA(cudaMemsetAsync(Mh.p, 0, Mh.bytes, s));
  LENS_CUDA(cudaMemsetAsync(Phi.p, 0, Phi.bytes, s));
  LENS_CUDA(cudaMemsetAsync(Psi.p, 0, Psi.bytes, s));
  AdjArgs A{};
  A.rays = rays; A.gy = gy;
  A.perm = RB.perm.as<int>(); A.ray_off = RB.off.as<int64_t>(); A.tile_off = RB.toff.as<int64_t>();
  A.nleaf = P.n_active_leaves;
  A.leaves = P.active_leaves; A.aidx = P.box_aidx; A.level = P.box_level; A.ix = P.box_ix;
  A.iy = P.box_iy; A.start = P.box_start; A.count = P.box_count; A.child = P.box_child;
  A.parent = P.box_parent;
  A.U_off = P.U_off; A.U_list = P.U_list; A.W_off = P.W_off; A.W_list = P.W_list;
  A.V_off = P.V_off; A.V_list = P.V_list; A.X_off = P.X_off; A.X_list = P.X_list;
  A.spos = P.spos; A.smass = P.smass; A.tab = P.tab;
  A.lo_x = P.root_lo[0]; A.lo_y = P.root_lo[1]; A.size = P.root_size; A.p = P.p;
  A.Lh = Lh.as<double2>(); A.Mh = Mh.as<double2>();
  A.Phi = Phi.as<double2>(); A.Psi = Psi.as<double2>();
  if (RB.total > (int64_t)INT32_MAX) fail(LENS_EINVAL, "too many rays in one adjoint call");
  if (RB.total > 0 && P.prec == LENS_FP32_BULK) {
    const size_t smem = sizeof(float2) * (size_t)P1 * 33;
    k_adj_leaf_moments32<<<(unsigned)RB.total, 32, smem, s>>>(A);
    LENS_LAUNCHED("k_adj_leaf_moments32");
    k_adj_p2p32<<<(unsigned)RB.total, 128, 0, s>>>(A);
    LENS_LAUNCHED("k_adj_p2p32");
  } else if (RB.total > 0) {
    const size_t smem = sizeof(double2) * (size_t)P1 * 32;
    if (smem > 48 * 1024)
      LENS_CUDA(cudaFuncSetAttribute(k_adj_leaf_moments, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    k_adj_leaf_moments<<<(unsigned)RB.total, 32, smem, s>>>(A);
    LENS_LAUNCHED("k_adj_leaf_moments");
    k_adj_p2p<<<(unsigned)RB.total, 128, 0, s>>>(A);
    LENS_LAUNCHED("k_adj_p2p");
  }
  // L2L^T, finest level first (levels >= 2 carry L2L)
  for (int l = P.nlevels - 1; l >= 2; --l) {
    const int64_t a0 = P.active_level_off[l], a1 = P.active_level_off[l + 1];
    if (a1 <= a0) continue;
    k_adj_l2l<<<grid_for((a1 - a0) * 32, 128), 128, 0, s>>>(A, P.active, a0, a1);
    LENS_LAUNCHED("k_adj_l2l");
  }
  if (P.n_active > 0) {
    k_adj_m2l<<<grid_for(P.n_active * 32, 128), 128, 0, s>>>(A, P.active, P.n_active);
    LENS_LAUNCHED("k_adj_m2l");
  }
  // M2M^T, coarsest level first
  for (int l = 1; l < P.nlevels; ++l) {
    const int64_t b0 = P.level_off[l], b1 = P.level_off[l + 1];
    k_adj_m2m<<<grid_for((b1 - b0) * 32, 128), 128, 0, s>>>(A, b0, b1);
    LENS_LAUNCHED("k_adj_m2m");
  }
  k_adj_p2m<<<grid_for(P.nb, 128), 128, 0, s>>>(A, P.nb);
  LENS_LAUNCHED("k_adj_p2m");
  if (gkg) {
    k_adj_kg<<<grid_for(m, 256, 1024), 256, 0, s>>>(rays, gy, m, gkg);
    LENS_LAUNCHED("k_adj_kg");
  }
  if (gxy || gm) {
    k_adj_out<<<grid_for(P.n, 256), 256, 0, s>>>(Phi.as<double2>(), Psi.as<double2>(), P.sidx, P.n,
                                                 gxy, gm);
    LENS_LAUNCHED("k_adj_out");
  }
}

}  // namespace lens
