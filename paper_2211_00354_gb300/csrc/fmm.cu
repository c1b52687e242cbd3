// fmm.cu -- upward and downward passes of the FMM in complex form
// (Appendix A: multipole "S" and local "R" expansions, the S2S/M2M, S2R/M2L
// and R2R/L2L translation theorems; Greengard & Rokhlin 1987).
//
// The Cauchy sum f(z) = sum_j m_j / (z - z_j) gives the deflection of Eq. 1
// as alpha = conj(f).  For a box of centre c and half-side r:
//   multipole  f(z) = sum_k a_k / (z-c)^(k+1),  a_k = sum_j m_j (z_j - c)^k,
//              stored scaled: A_k = a_k / r^k;
//   local      f(z) = sum_l b_l (z-c)^l,        stored scaled: B_l = b_l r^l.
// Scaled, the child->parent M2M and parent->child L2L matrices do not depend
// on the level (child offset = (+-1 +-i) r_parent / 2), and the M2L matrix of
// two same-level boxes depends only on their integer offset:
//   M2M  A^P_l = sum_{k<=l} C(l,k) 2^-k d^(l-k) A^C_k,       d = (+-1 +-i)/2
//   L2L  B^C_j = sum_{l>=j} C(l,j) 2^-j d^(l-j) B^P_l
//   M2L  B_l  += (-1)^l u^(l+1) / r * sum_k C(k+l,k) u^k A_k,  u = r/(c_B - c_C)
// The M2L is split into a diagonal pre-scaling (u^k), one REAL binomial
// matrix applied to the complex vector, and a diagonal post-scaling, which
// halves the float64 multiply-adds of a dense complex matrix.
//   P2L  B_l  += -(m / (z-c)) (r / (z-c))^l        (X lists)
// Every step here is float64 (the precision split keeps translations in
// float64).  On GB300 the float64 pipe is ~60x slower than float32, so these
// kernels are written to issue as few DFMAs as the series allow.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cx.cuh"
#include "lens_internal.h"

namespace lens {

namespace {

constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ double2 ld2(const double2* p) { return __ldg(p); }

// ---- P2M: one thread per leaf, accumulators in shared memory -----------------
// Leaves sorted by star count (counting sort, largest first), so that the
// lanes of a P2M warp run loops of equal length: with leaves of 1..leaf_size
// stars in tree order a warp would run its longest leaf's loop on all lanes.
// PASS 0 counts the non-empty leaves per star count and zeroes the expansions
// of empty leaves; PASS 1 places each leaf at offs[count] + rank.
template <int PASS>
__global__ void k_leaf_bins(const int* __restrict__ count, const int* __restrict__ child,
                            int64_t nb, int p, int leaf_size, int* __restrict__ bins,
                            int* __restrict__ offs, int* __restrict__ list,
                            double2* __restrict__ M) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int key = -1;
  if (b < nb && child[b] < 0) {
    const int nst = count[b];
    if (nst > 0) {
      key = min(nst, leaf_size);  // a leaf holds at most leaf_size stars
    } else if (PASS == 0) {
      double2* out = M + b * (int64_t)(p + 1);
      for (int k = 0; k <= p; ++k) out[k] = make_double2(0.0, 0.0);
    }
  }
  // one atomic per distinct count in the warp
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (key > 0 && lane == leader) base = atomicAdd(&bins[key], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (PASS == 1 && key > 0) list[offs[key] + base + __popc(peers & ((1u << lane) - 1u))] = (int)b;
}

// offs[k] for counts k = leaf_size .. 1 (descending), offs[0] = total
__global__ void k_bin_offsets(const int* __restrict__ bins, int leaf_size, int* __restrict__ offs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int acc = 0;
  for (int k = leaf_size; k >= 1; --k) { offs[k] = acc; acc += bins[k]; }
  offs[0] = acc;
}

// P2M: a_k = sum_j m_j w_j^k, w_j = (z_j - c)/r, into shared-memory
// accumulators [(p+1)][blockDim.x].  V = double2, or float2 for a float32-bulk
// plan: there the multipoles only feed far-field terms evaluated to float32
// accuracy, P2M is not one of the translations kept in float64, and the
// float64 pipe (~60x slower) would otherwise hold the upward pass on the
// build's critical path; w_j is formed in float64 and rounded once.
template <typename V>
__global__ void k_p2m(const double2* __restrict__ spos, const double* __restrict__ smass,
                      const int* __restrict__ start, const int* __restrict__ count,
                      const int* __restrict__ level, const int* __restrict__ ix,
                      const int* __restrict__ iy, const int* __restrict__ list,
                      const int* __restrict__ total, double lo_x, double lo_y, double root_size,
                      int p, double2* __restrict__ M) {
  extern __shared__ unsigned char acc_raw[];
  V* acc = reinterpret_cast<V*>(acc_raw);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= *total) return;
  const int64_t b = list[i];
  const int nst = count[b];
  double2* out = M + b * (int64_t)(p + 1);
  const double r = root_size / (double)(2ull << level[b]);
  const double cx = lo_x + (2.0 * ix[b] + 1.0) * r, cy = lo_y + (2.0 * iy[b] + 1.0) * r;
  const double ir = 1.0 / r;
  V* a = acc + threadIdx.x;
  const int st = blockDim.x;
  V zero;
  zero.x = 0; zero.y = 0;
  for (int k = 0; k <= p; ++k) a[k * st] = zero;
  const int s0 = start[b];
  for (int j = 0; j < nst; ++j) {
    const double2 z = spos[s0 + j];
    const double m = smass[s0 + j];
    V w, pw;
    w.x = (z.x - cx) * ir; w.y = (z.y - cy) * ir;
    pw.x = m; pw.y = 0;
    for (int k = 0; k <= p; ++k) {
      a[k * st] = a[k * st] + pw;
      pw = cmul(pw, w);
    }
  }
  for (int k = 0; k <= p; ++k) out[k] = make_double2(a[k * st].x, a[k * st].y);
}

// ---- M2M: one thread per (internal box, coefficient) of a level -------------
// The four child offsets are d_q = w i^m_q with w = (1+i)/2 and m_q = 2, 3,
// 1, 0 for quadrants (-,-), (+,-), (-,+), (+,+).  Since d_q^(l-k) depends on
// q only through i^(m_q (l-k)), which repeats with period 4 in l-k,
//   A^P_l = w^l sum_{k<=l} C(l,k) conj(w)^k G_{(l-k) mod 4}[k],
//   G_r[k] = sum_m i^(m r) A^(child m)_k      (a 4-point DFT over quadrants:
//                                              additions only),
// one REAL binomial matrix on four complex vectors instead of four complex
// matrices: about a third of the float64 operations of the direct form.
// w^k and conj(w)^k are exact, so the rounding is that of the direct form.
// Thread (parent, k) forms the four H_r[k] = conj(w)^k G_r[k], then thread
// (parent, l) sums row l: many short float64 chains instead of one long one
// per parent, so the pipe is fed from many warps.  A level's parents are
// walked through their children: the boxes of level l+1 are the groups of
// four children of the level-l splits, so group g (boxes c0+4g .. c0+4g+3)
// has one parent and no thread lands on a leaf.
constexpr int kM2MThreads = 128;

__global__ void __launch_bounds__(kM2MThreads)
k_m2m(const int* __restrict__ parent, int64_t c0, int64_t ngroups, int p,
      const double* __restrict__ binom, int ldb, const double2* __restrict__ wpow,
      double2* __restrict__ M) {
  extern __shared__ double2 H[];  // [parents per block][4][p+1], then the binomials
  const int P1 = p + 1;
  const int per = kM2MThreads / P1;  // parents per block (>= 1 for p <= 64)
  const int t = threadIdx.x, pb = t / P1, k = t - pb * P1;
  // rows 0..p of the binomial table, triangular (row l from l (l+1) / 2), in
  // shared memory: the row sums below then wait on no global load (a small
  // level has too few blocks to keep the table in L1)
  double* cb_tab = reinterpret_cast<double*>(H + (int64_t)per * 4 * P1);
  for (int i = t; i < P1 * (P1 + 1) / 2; i += kM2MThreads) {
    // i = l (l+1)/2 + kk, 0 <= kk <= l
    int l = (int)((sqrtf(8.f * (float)i + 1.f) - 1.f) * 0.5f);
    while (l * (l + 1) / 2 > i) --l;
    while ((l + 1) * (l + 2) / 2 <= i) ++l;
    cb_tab[i] = binom[(int64_t)l * ldb + (i - l * (l + 1) / 2)];
  }
  const int64_t g = (int64_t)blockIdx.x * per + pb;
  const bool on = pb < per && g < ngroups;
  const int64_t c = c0 + 4 * g;     // first child of the group
  const int64_t b = on ? parent[c] : 0;
  double2* Hp = H + (int64_t)pb * 4 * P1;
  if (on) {
    const double2* A = M + c * P1;  // children c .. c+3 are contiguous
    const double2 B0 = ld2(A + 3 * P1 + k), B1 = ld2(A + 2 * P1 + k);
    const double2 B2 = ld2(A + k), B3 = ld2(A + P1 + k);
    const double2 s02 = B0 + B2, d02 = B0 - B2, s13 = B1 + B3, d13 = B1 - B3;
    double2 w = ld2(wpow + k);
    w.y = -w.y;
    Hp[0 * P1 + k] = cmul(w, s02 + s13);
    Hp[1 * P1 + k] = cmul(w, make_double2(d02.x - d13.y, d02.y + d13.x));
    Hp[2 * P1 + k] = cmul(w, s02 - s13);
    Hp[3 * P1 + k] = cmul(w, make_double2(d02.x + d13.y, d02.y - d13.x));
  }
  __syncthreads();
  if (on) {
    const int l = k;
    double sx = 0.0, sy = 0.0;
    const double* crow = cb_tab + l * (l + 1) / 2;
    for (int kk = 0; kk <= l; ++kk) {
      const double cb = crow[kk];
      const double2 h = Hp[((l - kk) & 3) * P1 + kk];
      sx = fma(cb, h.x, sx);
      sy = fma(cb, h.y, sy);
    }
    M[b * (int64_t)P1 + l] = cmul(ld2(wpow + l), make_double2(sx, sy));
  }
}

// ---- downward pass ---------------------------------------------------------
// The far-field part of each local expansion (M2L over the V list, P2L over
// the X list) reads only multipole expansions and stars, so one launch forms
// it for the active boxes of every level at once, one warp per box: the
// float64 work of the coarse levels, a few boxes each, spreads over the whole
// GPU instead of a handful of SMs per level.  L2L, the only level-to-level
// dependence, then runs level by level from the top, one thread per
// (box, coefficient).
struct DownArgs {
  const int* active;
  int64_t a0, a1;
  const int* parent; const int* child; const int* level; const int* ix; const int* iy;
  const int* start; const int* count;
  const int64_t* V_off; const int* V_list;
  const int64_t* X_off; const int* X_list;
  const double2* spos; const double* smass;
  const double2* M;
  double2* L;
  FmmTables tab;
  double lo_x, lo_y, root_size;
  int p;
  int group;         // V entries per M2L pass
  size_t smem_warp;  // shared bytes per warp (multiple of 16)
};

// V entries per M2L pass: 32, fewer for large p so that a warp's buffers
// (2 G (p+1) complex values) stay within 24 KB.
inline int downward_group(int p) { return std::max(1, std::min(32, 24576 / (32 * (p + 1)))); }
// Shared bytes per warp: the larger of the P2L buffer ((p+1) x 32 complex +
// 64 ints) and the M2L buffers (2 G (p+1) complex + G ints).
inline size_t downward_smem_per_warp(int p) {
  const size_t p2l = sizeof(double2) * (size_t)(p + 1) * 32 + 64 * sizeof(int);
  const size_t g = (size_t)downward_group(p);
  const size_t m2l = sizeof(double2) * 2 * g * (size_t)(p + 1) + g * sizeof(int);
  return (std::max(p2l, m2l) + 15) / 16 * 16;
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_far_local(DownArgs A) {
  extern __shared__ double2 dsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t a = A.a0 + (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  if (a >= A.a1) return;
  const int p = A.p, P1 = p + 1;
  const int B = A.active[a];
  const int lv = A.level[B];
  const double r = A.root_size / (double)(2ull << lv);
  const double ir = 1.0 / r;
  double2 acc[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) acc[s] = make_double2(0.0, 0.0);
  // M2L from V.  Up to G entries at a time, their (entry, coefficient) pairs
  // spread over the lanes (p + 1 = 17 coefficients would leave 15 of 32 lanes
  // idle with one entry per pass):
  //   H[e][k] = A_k u_e^k                       (pre-scale)
  //   T[e][l] = (-1)^l u_e^(l+1) / r * sum_k C(k+l, k) H[e][k]
  //   B_l    += sum_e T[e][l]
  double2* buf = dsm + (int64_t)wib * (A.smem_warp / sizeof(double2));
  const int G = A.group;
  double2* H = buf;
  double2* T = buf + (int64_t)G * P1;
  int* uo = reinterpret_cast<int*>(T + (int64_t)G * P1);  // [G] offset-table rows
  const int bx = A.ix[B], by = A.iy[B];
  for (int64_t eb = A.V_off[a]; eb < A.V_off[a + 1]; eb += G) {
    const int ne = (int)min64(G, A.V_off[a + 1] - eb);
    for (int e = lane; e < ne; e += 32) {
      const int C = A.V_list[eb + e];
      uo[e] = ((A.iy[C] - by + 3) * 7 + (A.ix[C] - bx + 3)) * (p + 2);
    }
    __syncwarp();
    const int ntask = ne * P1;
    for (int t = lane; t < ntask; t += 32) {
      const int e = t / P1, k = t - e * P1;
      const int C = A.V_list[eb + e];
      H[t] = cmul(ld2(A.M + (int64_t)C * P1 + k), ld2(A.tab.upow + uo[e] + k));
    }
    __syncwarp();
    for (int t = lane; t < ntask; t += 32) {
      const int e = t / P1, l = t - e * P1;
      const double2* He = H + e * P1;
      double sx = 0.0, sy = 0.0;
      for (int k = 0; k <= p; ++k) {
        // C(k+l, k) = binom[(k+l)*ldb + k]
        const double c = __ldg(A.tab.binom + (int64_t)(k + l) * A.tab.ldb + k);
        const double2 v = He[k];
        sx = fma(c, v.x, sx);
        sy = fma(c, v.y, sy);
      }
      double2 post = ld2(A.tab.upow + uo[e] + l + 1);
      if (l & 1) post = make_double2(-post.x, -post.y);
      T[t] = cmul(post, make_double2(sx * ir, sy * ir));
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int l = lane + 32 * s;
      if (l > p) break;
      double2 v = acc[s];
      for (int e = 0; e < ne; ++e) v = v + T[e * P1 + l];
      acc[s] = v;
    }
    __syncwarp();
  }
  // P2L from X.  The stars of the X boxes are taken 32 at a time across box
  // boundaries: lane j forms the series -m_j/(z_j-c) (r/(z_j-c))^l of its
  // star by recurrence into shared memory, then lane l sums column l.  (One
  // star at a time with per-lane powers would idle most of the warp when the
  // X boxes hold a few stars each.)
  const double cx = A.lo_x + (2.0 * bx + 1.0) * r, cy = A.lo_y + (2.0 * by + 1.0) * r;
  int* xs = reinterpret_cast<int*>(buf + (int64_t)P1 * 32);  // [32] inclusive counts, [32] starts
  for (int64_t eb = A.X_off[a]; eb < A.X_off[a + 1]; eb += 32) {
    const int ne = (int)min64(32, A.X_off[a + 1] - eb);
    int cnt = 0, st = 0;
    if (lane < ne) {
      const int C = A.X_list[eb + lane];
      cnt = A.count[C];
      st = A.start[C];
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    xs[lane] = incl;
    xs[32 + lane] = st;
    __syncwarp();
    for (int f0 = 0; f0 < total; f0 += 32) {
      const int f = f0 + lane;
      if (f < total) {
        int e = 0;
        while (xs[e] <= f) ++e;  // first box whose inclusive count exceeds f
        const int j = xs[32 + e] + f - (e ? xs[e - 1] : 0);
        const double2 z = A.spos[j];
        const double m = A.smass[j];
        const double2 inv = cinv(make_double2(z.x - cx, z.y - cy));  // 1/(z-c)
        const double2 q = make_double2(inv.x * r, inv.y * r);        // r/(z-c)
        double2 v = make_double2(-m * inv.x, -m * inv.y);            // -m/(z-c)
        for (int l = 0; l <= p; ++l) {
          buf[l * 32 + lane] = v;
          v = cmul(v, q);
        }
      }
      __syncwarp();
      const int nv = min(32, total - f0);
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const int l = lane + 32 * s;
        if (l > p) break;
        double2 v = acc[s];
        for (int jj = 0; jj < nv; ++jj) v = v + buf[l * 32 + jj];
        acc[s] = v;
      }
      __syncwarp();
    }
  }
  double2* out = A.L + (int64_t)B * P1;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int l = lane + 32 * s;
    if (l <= p) out[l] = acc[s];
  }
}

// L2L of the active boxes of one level (>= 2; above it the parent's local
// expansion is zero), one thread per (box, coefficient j):
//   L_B[j] += sum_{l >= j} S_q[j][l] L_parent[l],  q = the box's quadrant.
// The parent of an active box is active and its expansion is final.
__global__ void k_l2l(const int* __restrict__ active, int64_t a0, int64_t a1,
                      const int* __restrict__ parent, const int* __restrict__ child,
                      const double2* __restrict__ l2l, int p, double2* __restrict__ L) {
  const int P1 = p + 1;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t a = a0 + t / P1;
  if (a >= a1) return;
  const int j = (int)(t - (a - a0) * P1);
  const int B = active[a];
  const int par = parent[B];
  const int q = B - child[par];
  const double2* Lp = L + (int64_t)par * P1;
  const double2* S = l2l + ((int64_t)q * P1 + j) * P1;
  double2 v = make_double2(0.0, 0.0);
  for (int l = j; l <= p; ++l) v = cfma(ld2(S + l), ld2(Lp + l), v);
  double2* o = L + (int64_t)B * P1 + j;
  *o = *o + v;
}

}  // namespace

// ---- host: tables ----------------------------------------------------------
void fmm_tables(Plan& P, cudaStream_t s) {
  const int p = P.p;
  const int P1 = p + 1;
  FmmTables& t = P.tab;
  t.p = p;
  t.ldb = p + 2;
  const int nb = 2 * p + 2;
  std::vector<double> bin((size_t)nb * t.ldb, 0.0);
  std::vector<std::vector<double>> full(nb, std::vector<double>(nb, 0.0));
  for (int n = 0; n < nb; ++n) {
    full[n][0] = 1.0;
    for (int k = 1; k <= n; ++k) full[n][k] = full[n - 1][k - 1] + (k <= n - 1 ? full[n - 1][k] : 0.0);
  }
  for (int n = 0; n < nb; ++n)
    for (int k = 0; k < t.ldb && k <= n; ++k) bin[(size_t)n * t.ldb + k] = full[n][k];
  auto cpow = [](double re, double im, int e) {
    double pr = 1.0, pi = 0.0;
    for (int i = 0; i < e; ++i) {
      double nr = pr * re - pi * im, ni = pr * im + pi * re;
      pr = nr; pi = ni;
    }
    return std::pair<double, double>(pr, pi);
  };
  std::vector<double2> m2m((size_t)4 * P1 * P1), l2l((size_t)4 * P1 * P1);
  for (int q = 0; q < 4; ++q) {
    const double dre = ((q & 1) ? 0.5 : -0.5), dim = ((q >> 1) ? 0.5 : -0.5);
    for (int l = 0; l <= p; ++l)
      for (int k = 0; k <= p; ++k) {
        double2 v = make_double2(0.0, 0.0);
        if (k <= l) {
          auto d = cpow(dre, dim, l - k);
          const double c = full[l][k] * std::ldexp(1.0, -k);
          v = make_double2(c * d.first, c * d.second);
        }
        m2m[((size_t)q * P1 + l) * P1 + k] = v;
      }
    for (int j = 0; j <= p; ++j)
      for (int l = 0; l <= p; ++l) {
        double2 v = make_double2(0.0, 0.0);
        if (l >= j) {
          auto d = cpow(dre, dim, l - j);
          const double c = full[l][j] * std::ldexp(1.0, -j);
          v = make_double2(c * d.first, c * d.second);
        }
        l2l[((size_t)q * P1 + j) * P1 + l] = v;
      }
  }
  std::vector<double2> up((size_t)49 * (p + 2));
  for (int dy = -3; dy <= 3; ++dy)
    for (int dx = -3; dx <= 3; ++dx) {
      const int o = (dy + 3) * 7 + (dx + 3);
      // u = r / (c_B - c_C) = -1 / (2 (dx + i dy))
      double ure = 0, uim = 0;
      if (dx != 0 || dy != 0) {
        const double den = 2.0 * (dx * (double)dx + dy * (double)dy);
        ure = -dx / den;
        uim = dy / den;
      }
      double pr = 1.0, pi = 0.0;
      for (int k = 0; k <= p + 1; ++k) {
        up[(size_t)o * (p + 2) + k] = make_double2(pr, pi);
        const double nr = pr * ure - pi * uim, ni = pr * uim + pi * ure;
        pr = nr; pi = ni;
      }
    }
  // ((1+i)/2)^k: Gaussian integers over powers of two, exact in float64
  std::vector<double2> wp((size_t)P1);
  for (int k = 0; k <= p; ++k) {
    auto w = cpow(0.5, 0.5, k);
    wp[(size_t)k] = make_double2(w.first, w.second);
  }
  // one host block (kept in the plan until the copy has run: no wait here);
  // bin holds (2p+2)(p+2) doubles, an even count, so the complex tables
  // after it start on 16-byte boundaries
  const size_t nd = bin.size() + 2 * (m2m.size() + l2l.size() + up.size() + wp.size());
  P.tab_host.assign(nd, 0.0);
  double* h = P.tab_host.data();
  std::memcpy(h, bin.data(), bin.size() * sizeof(double));
  size_t o = bin.size();
  for (const auto* v : {&m2m, &l2l, &up, &wp}) {
    std::memcpy(h + o, v->data(), v->size() * sizeof(double2));
    o += 2 * v->size();
  }
  double* d = P.dalloc_n<double>(nd);
  LENS_CUDA(cudaMemcpyAsync(d, h, nd * sizeof(double), cudaMemcpyHostToDevice, s));
  o = bin.size();
  t.binom = d;
  t.m2m = reinterpret_cast<double2*>(d + o); o += 2 * m2m.size();
  t.l2l = reinterpret_cast<double2*>(d + o); o += 2 * l2l.size();
  t.upow = reinterpret_cast<double2*>(d + o); o += 2 * up.size();
  t.wpow = reinterpret_cast<double2*>(d + o);
}

void fmm_alloc(Plan& P) {
  const size_t P1 = (size_t)P.p + 1;
  if (!P.M) P.M = P.dalloc_n<double2>((size_t)P.nb * P1);
  if (!P.L) P.L = P.dalloc_n<double2>((size_t)P.nb * P1);
  if (!P.p2m_list) P.p2m_list = P.dalloc_n<int>((size_t)P.nb);
  if (!P.p2m_bins) P.p2m_bins = P.dalloc_n<int>(2 * ((size_t)P.leaf + 1));
}

void fmm_p2m(Plan& P, cudaStream_t s) {
  const int p = P.p, P1 = p + 1;
  if (!P.M || !P.p2m_list || !P.p2m_bins) fail(LENS_ECUDA, "internal: expansion buffers not allocated");
  // P2M on every non-empty leaf (thread per leaf, leaves sorted by star
  // count), all levels at once
  const int L = P.leaf;
  int* cnt = P.p2m_bins;
  int* offs = cnt + (L + 1);
  int* list = P.p2m_list;
  LENS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(L + 1), s));
  k_leaf_bins<0><<<grid_for(P.nb, 256), 256, 0, s>>>(P.box_count, P.box_child, P.nb, p, L, cnt, offs,
                                                      list, P.M);
  LENS_LAUNCHED("k_leaf_bins<count>");
  k_bin_offsets<<<1, 32, 0, s>>>(cnt, L, offs);
  LENS_LAUNCHED("k_bin_offsets");
  LENS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(L + 1), s));
  k_leaf_bins<1><<<grid_for(P.nb, 256), 256, 0, s>>>(P.box_count, P.box_child, P.nb, p, L, cnt, offs,
                                                      list, P.M);
  LENS_LAUNCHED("k_leaf_bins<place>");
  const int tpb = 32;
  if (P.prec == LENS_FP32_BULK) {
    const size_t smem = sizeof(float2) * (size_t)P1 * tpb;
    if (smem > 48 * 1024)
      LENS_CUDA(cudaFuncSetAttribute(k_p2m<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    k_p2m<float2><<<grid_for(P.nb, tpb), tpb, smem, s>>>(
        P.spos, P.smass, P.box_start, P.box_count, P.box_level, P.box_ix, P.box_iy, list, offs,
        P.root_lo[0], P.root_lo[1], P.root_size, p, P.M);
  } else {
    const size_t smem = sizeof(double2) * (size_t)P1 * tpb;
    if (smem > 48 * 1024)
      LENS_CUDA(cudaFuncSetAttribute(k_p2m<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    k_p2m<double2><<<grid_for(P.nb, tpb), tpb, smem, s>>>(
        P.spos, P.smass, P.box_start, P.box_count, P.box_level, P.box_ix, P.box_iy, list, offs,
        P.root_lo[0], P.root_lo[1], P.root_size, p, P.M);
  }
  LENS_LAUNCHED("k_p2m");
}

void fmm_m2m(Plan& P, cudaStream_t s) {
  const FmmTables& t = P.tab;
  const int P1 = P.p + 1;
  const int per = kM2MThreads / P1;
  const size_t smem = sizeof(double2) * 4 * (size_t)P1 * per + sizeof(double) * P1 * (P1 + 1) / 2;
  for (int l = P.nlevels - 2; l >= 0; --l) {
    // level l+1 holds the children of the level-l splits, four per split
    const int64_t c0 = P.level_off[l + 1], ng = (P.level_off[l + 2] - c0) / 4;
    if (ng <= 0) continue;
    k_m2m<<<grid_for(ng, per), kM2MThreads, smem, s>>>(P.box_parent, c0, ng, P.p, t.binom,
                                                       t.ldb, t.wpow, P.M);
    LENS_LAUNCHED("k_m2m");
  }
}

void fmm_downward(Plan& P, cudaStream_t s) {
  const FmmTables& t = P.tab;
  if (!P.L) P.L = P.dalloc_n<double2>((size_t)P.nb * (P.p + 1));
  DownArgs A{};
  A.active = P.active;
  A.parent = P.box_parent; A.child = P.box_child; A.level = P.box_level;
  A.ix = P.box_ix; A.iy = P.box_iy; A.start = P.box_start; A.count = P.box_count;
  A.V_off = P.V_off; A.V_list = P.V_list; A.X_off = P.X_off; A.X_list = P.X_list;
  A.spos = P.spos; A.smass = P.smass; A.M = P.M; A.L = P.L; A.tab = t;
  A.lo_x = P.root_lo[0]; A.lo_y = P.root_lo[1]; A.root_size = P.root_size; A.p = P.p;
  A.group = downward_group(P.p);
  A.smem_warp = downward_smem_per_warp(P.p);
  const size_t smem = A.smem_warp * kWarpsPerBlock;
  if (smem > 48 * 1024)
    LENS_CUDA(cudaFuncSetAttribute(k_far_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  A.a0 = 0;
  A.a1 = P.n_active;
  if (A.a1 > 0) {
    if (P.ev_far0) LENS_CUDA(cudaEventRecord(P.ev_far0, s));
    k_far_local<<<grid_for(A.a1 * 32, 32 * kWarpsPerBlock), 32 * kWarpsPerBlock, smem, s>>>(A);
    LENS_LAUNCHED("k_far_local");
    if (P.ev_far1) LENS_CUDA(cudaEventRecord(P.ev_far1, s));
  }
  const int P1 = P.p + 1;
  for (int l = 2; l < P.nlevels; ++l) {
    const int64_t a0 = P.active_level_off[l], a1 = P.active_level_off[l + 1];
    if (a1 <= a0) continue;
    k_l2l<<<grid_for((a1 - a0) * P1, 128), 128, 0, s>>>(P.active, a0, a1, P.box_parent,
                                                       P.box_child, t.l2l, P.p, P.L);
    LENS_LAUNCHED("k_l2l");
  }
}

}  // namespace lens
