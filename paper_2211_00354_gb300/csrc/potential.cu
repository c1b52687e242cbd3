// potential.cu -- the lensing potential psi(x) = sum_i m_i ln|x - x_i| +
// kappa_s |x|^2 / 2 + gamma (x1^2 - x2^2) / 2, whose gradient is x - y
// (Eq. 1 with its smooth field), through the plan's expansions (the
// potential of Sec. 2.5's lens; Appendix A's expansions of the complex
// logarithm, Greengard & Rokhlin 1987).
//
// With Phi(z) = sum_j m_j log(z - z_j), psi = Re Phi + smooth, and Phi' = f,
// the Cauchy sum the plan expands.  So the potential needs no new
// expansions, only their integrals and one real constant per box:
//   multipole  Phi(z) = a_0 log(z-c) - sum_{k>=1} a_k / (k (z-c)^k)
//   local      Phi(z) = c_B + sum_l b_l (z-c)^(l+1) / (l+1)
// (a_k, b_l the plan's field coefficients; stored scaled, A_k = a_k / r^k,
// B_l = b_l r^l).  The constant c_B = Re Phi_far(c_B) collects
//   M2L  over V:  a_0 ln|t| - Re sum_{k>=1} (A_k / k) u^k,  t = c_B - c_C, u = r / t
//   P2L  over X:  sum_j m_j ln|c_B - z_j|
//   L2L  from the parent P:  c_P + r_P Re sum_l B^P_l d^(l+1) / (l+1),
//        d = (c_B - c_P) / r_P = (+-1 +-i) / 2
// and a ray z in leaf B (half-side r, w = (z - c_B) / r) gets
//   L2P  c_B + r Re sum_l B_l w^(l+1) / (l+1)
//   P2P  over U (the leaf itself included): sum_j m_j ln|z - z_j| (a star
//        exactly at the ray contributes nothing)
//   M2P  over W:  a_0 ln|z - c_C| - Re sum_{k>=1} (A_k / k) (r_C / (z - c_C))^k
// All float64; a thread per ray descends the tree to its leaf, the rays taken
// in leaf order (bucketed as the deflection's ray path does), so that the
// lanes of a warp share their leaf's lists and stars.  Divisions by
// the small integers k take a per-block table of 1/k, and with equal masses
// the near field's logarithms are taken of products of up to 8 squared
// distances (flushed early outside [1e-200, 1e200]): one float64 log where
// there were eight, on GB300's slow float64 pipe.
#include "cx.cuh"
#include "potential.h"

namespace lens {
namespace {

struct PotArgs {
  int p;
  double lo_x, lo_y, size;
  int depth;
  const int* level; const int* ix; const int* iy; const int* parent; const int* child;
  const int* aidx; const int* lidx; const int* start; const int* count; const int* active;
  const double2* spos; const double* smass;
  const double2* M; const double2* L;
  const int64_t* V_off; const int* V_list; const int64_t* X_off; const int* X_list;
  const int64_t* U_off; const int* U_list; const int64_t* W_off; const int* W_list;
  double* c0;  // per active box
  double ks, g;
  int um;        // all masses equal to m0
  double m0;
};

__device__ __forceinline__ double half_side(const PotArgs& A, int level) {
  return A.size / (double)(2ull << level);
}
__device__ __forceinline__ double2 centre(const PotArgs& A, int b, double r) {
  return make_double2(A.lo_x + (2.0 * A.ix[b] + 1.0) * r, A.lo_y + (2.0 * A.iy[b] + 1.0) * r);
}
// -Re sum_{k=1..p} (A_k / k) v^k, inv[k] = 1/k
__device__ __forceinline__ double tail(const double2* Ak, int p, double2 v, const double* inv) {
  double s = 0.0;
  double2 pw = v;
  for (int k = 1; k <= p; ++k) {
    s -= (Ak[k].x * pw.x - Ak[k].y * pw.y) * inv[k];
    pw = cmul(pw, v);
  }
  return s;
}

// 1/k for k = 0 .. n-1 in shared memory (1/0 unused); block-cooperative
constexpr int kPotInv = kMaxOrder + 2;
__device__ __forceinline__ void fill_inv(double* inv, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) inv[k] = k ? 1.0 / (double)k : 0.0;
  __syncthreads();
}

// own constant of every active box: M2L over V and P2L over X (warp per box)
__global__ void k_pot_own(PotArgs A, int64_t nact) {
  __shared__ double inv[kPotInv];
  fill_inv(inv, A.p + 2);
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= nact) return;
  const int B = A.active[a];
  const double r = half_side(A, A.level[B]);
  const double2 cB = centre(A, B, r);
  const int P1 = A.p + 1;
  double acc = 0.0;
  for (int64_t e = A.V_off[a] + lane; e < A.V_off[a + 1]; e += 32) {
    const int C = A.V_list[e];
    const double2 cC = centre(A, C, r);
    const double2 t = make_double2(cB.x - cC.x, cB.y - cC.y);
    const double2* Ak = A.M + (int64_t)C * P1;
    const double2 it = cinv(t);
    acc += Ak[0].x * 0.5 * log(t.x * t.x + t.y * t.y) +
           tail(Ak, A.p, make_double2(r * it.x, r * it.y), inv);
  }
  for (int64_t e = A.X_off[a]; e < A.X_off[a + 1]; ++e) {
    const int C = A.X_list[e];
    for (int j = A.start[C] + lane; j < A.start[C] + A.count[C]; j += 32) {
      const double dx = cB.x - A.spos[j].x, dy = cB.y - A.spos[j].y;
      acc += A.smass[j] * 0.5 * log(dx * dx + dy * dy);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) A.c0[a] = acc;
}

// the parent's far field at each box centre, one level at a time (thread per
// active box of the level)
__global__ void k_pot_down(PotArgs A, int64_t a0, int64_t a1) {
  const int64_t a = a0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= a1) return;
  const int B = A.active[a];
  const int Pb = A.parent[B];
  if (Pb < 0) return;
  const int ap = A.aidx[Pb];
  if (ap < 0) return;
  const double rP = half_side(A, A.level[Pb]);
  const double2 d = make_double2((2.0 * A.ix[B] + 1.0 - 2.0 * (2.0 * A.ix[Pb] + 1.0)) * 0.5,
                                 (2.0 * A.iy[B] + 1.0 - 2.0 * (2.0 * A.iy[Pb] + 1.0)) * 0.5);
  const double2* Bl = A.L + (int64_t)Pb * (A.p + 1);
  // sum_l B_l d^(l+1) / (l+1) by Horner
  double2 acc = make_double2(Bl[A.p].x / (A.p + 1), Bl[A.p].y / (A.p + 1));
  for (int l = A.p - 1; l >= 0; --l) {
    acc = cmul(acc, d);
    acc.x += Bl[l].x / (l + 1);
    acc.y += Bl[l].y / (l + 1);
  }
  acc = cmul(acc, d);
  A.c0[a] += A.c0[ap] + rP * acc.x;
}

__global__ void k_pot_eval(PotArgs A, const double* __restrict__ rays, int64_t m,
                           const int* __restrict__ perm, double* __restrict__ psi,
                           int* __restrict__ err) {
  __shared__ double inv[kPotInv];
  fill_inv(inv, A.p + 2);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m) return;
  const int64_t r = perm[t];
  const double x = rays[2 * r], y = rays[2 * r + 1];
  const double scale = (double)(1ull << A.depth) / A.size;
  const double qmax = (double)((1u << A.depth) - 1u);
  const double fx = floor((x - A.lo_x) * scale), fy = floor((y - A.lo_y) * scale);
  if (!(fx >= 0.0 && fx <= qmax && fy >= 0.0 && fy <= qmax)) {  // also catches NaN
    atomicExch(err, 1);
    psi[r] = NAN;
    return;
  }
  const uint32_t qx = (uint32_t)fx, qy = (uint32_t)fy;
  int b = 0;
  for (int l = 0; l < A.depth; ++l) {
    const int c = A.child[b];
    if (c < 0) break;
    const int sh = A.depth - l - 1;
    b = c + (int)(((qx >> sh) & 1u) | (((qy >> sh) & 1u) << 1));
  }
  const int a = A.aidx[b];
  if (A.lidx[b] < 0 || a < 0) {
    atomicExch(err, 1);
    psi[r] = NAN;
    return;
  }
  const double rb = half_side(A, A.level[b]);
  const double2 cb = centre(A, b, rb);
  const int P1 = A.p + 1;
  // L2P of the integrated local expansion
  const double2 w = make_double2((x - cb.x) / rb, (y - cb.y) / rb);
  const double2* Bl = A.L + (int64_t)b * P1;
  double2 acc = make_double2(Bl[A.p].x * inv[P1], Bl[A.p].y * inv[P1]);
  for (int l = A.p - 1; l >= 0; --l) {
    acc = cmul(acc, w);
    acc.x += Bl[l].x * inv[l + 1];
    acc.y += Bl[l].y * inv[l + 1];
  }
  acc = cmul(acc, w);
  double phi = A.c0[a] + rb * acc.x;
  // P2P over U (a star exactly at the ray contributes nothing)
  if (A.um) {
    double lsum = 0.0, prod = 1.0;
    int n = 0;
    for (int64_t e = A.U_off[a]; e < A.U_off[a + 1]; ++e) {
      const int C = A.U_list[e];
      for (int j = A.start[C]; j < A.start[C] + A.count[C]; ++j) {
        const double dx = x - A.spos[j].x, dy = y - A.spos[j].y;
        const double d2 = dx * dx + dy * dy;
        if (!(d2 > 0.0)) continue;
        prod *= d2;
        if (++n == 8 || !(prod > 1e-200 && prod < 1e200)) {
          lsum += log(prod);
          prod = 1.0;
          n = 0;
        }
      }
    }
    if (n > 0) lsum += log(prod);
    phi += 0.5 * A.m0 * lsum;
  } else {
    for (int64_t e = A.U_off[a]; e < A.U_off[a + 1]; ++e) {
      const int C = A.U_list[e];
      for (int j = A.start[C]; j < A.start[C] + A.count[C]; ++j) {
        const double dx = x - A.spos[j].x, dy = y - A.spos[j].y;
        const double d2 = dx * dx + dy * dy;
        if (d2 > 0.0) phi += A.smass[j] * 0.5 * log(d2);
      }
    }
  }
  // M2P over W
  for (int64_t e = A.W_off[a]; e < A.W_off[a + 1]; ++e) {
    const int C = A.W_list[e];
    const double rC = half_side(A, A.level[C]);
    const double2 cC = centre(A, C, rC);
    const double2 t = make_double2(x - cC.x, y - cC.y);
    const double2* Ak = A.M + (int64_t)C * P1;
    const double2 it = cinv(t);
    phi += Ak[0].x * 0.5 * log(t.x * t.x + t.y * t.y) +
           tail(Ak, A.p, make_double2(rC * it.x, rC * it.y), inv);
  }
  psi[r] = phi + 0.5 * A.ks * (x * x + y * y) + 0.5 * A.g * (x * x - y * y);
}

}  // namespace

void evaluate_potential(Plan& P, const double* rays, int64_t m, double* psi, cudaStream_t s) {
  if (m == 0) return;
  if (P.n_active == 0) fail(LENS_EDOMAIN, "plan has no active boxes");
  // the rays in leaf order (fails with LENS_EDOMAIN for a ray outside the root)
  RayBuckets RB;
  bucket_rays(P, rays, m, 1, RB, s);
  wait_expansions(P, s);
  Scratch c0(&P.da, sizeof(double) * (size_t)P.n_active);
  Scratch err(&P.da, sizeof(int));
  LENS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  PotArgs A{};
  A.p = P.p;
  A.lo_x = P.root_lo[0]; A.lo_y = P.root_lo[1]; A.size = P.root_size; A.depth = P.depth;
  A.level = P.box_level; A.ix = P.box_ix; A.iy = P.box_iy; A.parent = P.box_parent;
  A.child = P.box_child; A.aidx = P.box_aidx; A.lidx = P.box_lidx; A.start = P.box_start;
  A.count = P.box_count; A.active = P.active; A.spos = P.spos; A.smass = P.smass;
  A.M = P.M; A.L = P.L;
  A.V_off = P.V_off; A.V_list = P.V_list; A.X_off = P.X_off; A.X_list = P.X_list;
  A.U_off = P.U_off; A.U_list = P.U_list; A.W_off = P.W_off; A.W_list = P.W_list;
  A.c0 = c0.as<double>();
  A.ks = P.kappa_s; A.g = P.gamma;
  A.um = P.equal_mass ? 1 : 0;
  A.m0 = P.mass0;
  k_pot_own<<<grid_for(P.n_active * 32, 256), 256, 0, s>>>(A, P.n_active);
  LENS_LAUNCHED("k_pot_own");
  for (size_t l = 1; l + 1 < P.active_level_off.size(); ++l) {
    const int64_t a0 = P.active_level_off[l], a1 = P.active_level_off[l + 1];
    if (a1 <= a0) continue;
    k_pot_down<<<grid_for(a1 - a0, 128), 128, 0, s>>>(A, a0, a1);
    LENS_LAUNCHED("k_pot_down");
  }
  k_pot_eval<<<grid_for(m, 128), 128, 0, s>>>(A, rays, m, RB.perm.as<int>(), psi, err.as<int>());
  LENS_LAUNCHED("k_pot_eval");
  int herr = 0;
  LENS_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaStreamSynchronize(s));
  if (herr) fail(LENS_EDOMAIN, "a ray lies outside the plan's target region (or is not finite)");
}

}  // namespace lens
