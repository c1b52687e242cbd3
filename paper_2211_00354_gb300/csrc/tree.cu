// tree.cu -- GPU quadtree over the stars and the adaptive FMM interaction
// lists (Appendix A, step 1: hierarchical four-fold partition of the plane).
//
// Build:
//  1. root square = bounding box of the stars united with the target region;
//  2. 56-bit Morton keys (28 levels) and an LSD radix sort of (key, index);
//  3. split-node enumeration: in Morton order, star i begins a node at every
//     level deeper than the common prefix it shares with star i-1; a node at
//     level l < depth splits iff it holds more than leaf_size stars (its end
//     comes from a binary search on the sorted keys).  One host sync reads the
//     per-level split counts, which fix every array size;
//  4. boxes are numbered level by level, Morton order within a level: the 4
//     children of the split node of rank k at level l are boxes
//     level_off[l+1] + 4k + q.  Empty quadrants stay as leaves, so the leaves
//     tile the root and any point has a leaf;
//  5. boxes that meet the target region are "active" (they get local
//     expansions); lists are built for active boxes only.
//
// Interaction lists of an active box B at level l (adaptive FMM, Carrier-
// Greengard-Rokhlin): V(B) = non-adjacent children of the parent's colleagues
// (M2L); X(B) = leaves coarser than B adjacent to the parent but not to B
// (P2L); for a leaf B also U(B) = adjacent leaves (P2P) and W(B) =
// non-adjacent children of adjacent boxes finer than B (M2P).  Empty boxes
// are skipped in every list.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cx.cuh"
#include "lens_internal.h"
#include "okey.cuh"

namespace lens {

namespace {

struct LevelOffsets {
  int64_t off[kMaxDepth + 2];
  int nlevels;
};

// per block: x min, x max, y min, y max, non-finite count, mass min, mass max
constexpr int kBoundsParts = 7;

// Per block: the bounds of its stars (grid-stride) by order-preserving
// integer keys (okey.cuh: exact, on the integer pipe), reduced by warp
// shuffles and across the block's warps.
constexpr int kBoundsThreads = 256;

__global__ void __launch_bounds__(kBoundsThreads)
k_bounds(const double* __restrict__ stars, const double* __restrict__ m, int64_t n,
         double* __restrict__ part) {
  constexpr int kW = kBoundsThreads / 32;
  __shared__ unsigned long long sh[6][kW];
  __shared__ unsigned int shb[kW];
  // keys of x min, x max, y min, y max, mass min, mass max
  unsigned long long k[6] = {~0ull, 0ull, ~0ull, 0ull, ~0ull, 0ull};
  unsigned int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = stars[2 * i], y = stars[2 * i + 1], w = m[i];
    if (!(finite_bits(x) && finite_bits(y) && finite_bits(w))) { ++bad; continue; }
    const unsigned long long kx = okey(x), ky = okey(y), kw = okey(w);
    k[0] = min(k[0], kx); k[1] = max(k[1], kx);
    k[2] = min(k[2], ky); k[3] = max(k[3], ky);
    k[4] = min(k[4], kw); k[5] = max(k[5], kw);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, k[q], o);
      k[q] = (q & 1) ? max(k[q], v) : min(k[q], v);
    }
  }
  bad = __reduce_add_sync(0xffffffffu, bad);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 6; ++q) sh[q][w] = k[q];
    shb[w] = bad;
  }
  __syncthreads();
  if (threadIdx.x < kBoundsParts) {
    const int t = threadIdx.x;
    double v;
    if (t == 4) {
      unsigned int s = 0;
      for (int q = 0; q < kW; ++q) s += shb[q];
      v = (double)s;
    } else {
      // slots 0..3 and 5, 6: the key row t (t < 4) or t - 1
      const int q = t < 4 ? t : t - 1;
      unsigned long long r = sh[q][0];
      for (int j = 1; j < kW; ++j) r = (q & 1) ? max(r, sh[q][j]) : min(r, sh[q][j]);
      // no finite star in this block: the empty bounds
      const bool none = (q & 1) ? r == 0ull : r == ~0ull;
      v = none ? ((q & 1) ? -INFINITY : INFINITY) : unkey(r);
    }
    part[blockIdx.x * kBoundsParts + t] = v;
  }
}

__global__ void k_keys(const double* __restrict__ stars, int64_t n, double lo_x, double lo_y,
                       double scale, int depth, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double qmax = (double)((1u << depth) - 1u);
  double fx = floor((stars[2 * i] - lo_x) * scale);
  double fy = floor((stars[2 * i + 1] - lo_y) * scale);
  fx = fmin(fmax(fx, 0.0), qmax);
  fy = fmin(fmax(fy, 0.0), qmax);
  keys[i] = morton((uint32_t)fx, (uint32_t)fy);
  idx[i] = (uint32_t)i;
}

__global__ void k_gather(const double* __restrict__ stars, const double* __restrict__ m,
                         const uint32_t* __restrict__ idx, int64_t n, double2* __restrict__ spos,
                         double* __restrict__ smass) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t j = idx[i];
  spos[i] = make_double2(stars[2 * (int64_t)j], stars[2 * (int64_t)j + 1]);
  smass[i] = m[j];
}

// first index in [lo, hi) whose key is > v  (keys sorted ascending)
__device__ __forceinline__ int64_t upper_bound(const uint64_t* k, int64_t lo, int64_t hi, uint64_t v) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (k[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t lower_bound(const uint64_t* k, int64_t lo, int64_t hi, uint64_t v) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (k[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int first_level(const uint64_t* k, int64_t i, int depth) {
  if (i == 0) return 0;
  const uint64_t x = k[i - 1] ^ k[i];
  if (x == 0) return depth + 1;
  const int lcp = (__clzll((long long)x) - (64 - 2 * depth)) >> 1;
  return lcp + 1;
}

// Pass 1 (write == false): per-level split counts, in total and per block
// (bcnt, level-major: bcnt[l * blocks + block]).  Pass 2: write the entries
// (level << 32 | first star) in star order within each level, which is the
// order of (level, box code) that k_fill_boxes reads: boff is the exclusive
// scan of bcnt (the level-major layout makes it the level's offset plus the
// entries of earlier blocks), and inside a block the entries of a level are
// ranked in thread order by warp ballots.  The grid is the same in both
// passes (kSplitThreads threads a block over the n stars).
// The keys need only be sorted by their level-dcap prefixes (the top 2 dcap
// of their 2 depth bits): a box of level dcap with more than leaf stars sets
// deep_flag (the caller then sorts fully, or, at dcap == depth, fails).
constexpr int kSplitThreads = 256;

template <bool WRITE>
__global__ void __launch_bounds__(kSplitThreads)
k_splits(const uint64_t* __restrict__ k, int64_t n, int depth, int dcap, int leaf,
         unsigned long long* __restrict__ counts, int* __restrict__ deep_flag,
         int64_t* __restrict__ bcnt, const int64_t* __restrict__ boff,
         uint64_t* __restrict__ out) {
  constexpr int kW = kSplitThreads / 32;
  __shared__ unsigned int sc[kMaxDepth + 1];
  __shared__ unsigned int wc[kMaxDepth][kW];
  __shared__ int lrange[2];
  for (int q = threadIdx.x; q <= kMaxDepth; q += blockDim.x) sc[q] = 0;
  if (threadIdx.x == 0) { lrange[0] = kMaxDepth; lrange[1] = -1; }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  uint64_t ki = 0, kl = 0;
  int l0 = depth + 1;
  if (i < n) {
    ki = k[i];
    // star i + leaf shares the level-l prefix exactly when the box starting
    // at i holds more than leaf stars (the keys are sorted by prefix)
    kl = i + leaf < n ? k[i + leaf] : ~ki;
    l0 = first_level(k, i, depth);
  }
  auto more = [&](int l) {
    return l == 0 ? n > leaf : i + leaf < n && ((ki ^ kl) >> (2 * (depth - l))) == 0;
  };
  // the levels at which the box starting at star i splits: l0 .. l1-1
  int l1 = l0;
  if (i < n) {
    for (; l1 <= depth && more(l1); ++l1) {
      if (l1 == dcap) {
        if (!WRITE) atomicExch(deep_flag, 1);
        break;
      }
    }
  }
  if constexpr (!WRITE) {
    for (int l = l0; l < l1; ++l) atomicAdd(&sc[l], 1u);
    __syncthreads();
    for (int q = threadIdx.x; q < kMaxDepth; q += blockDim.x) {
      if (sc[q]) atomicAdd(&counts[q], (unsigned long long)sc[q]);
      bcnt[(int64_t)q * gridDim.x + blockIdx.x] = sc[q];
    }
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (l1 > l0) { atomicMin(&lrange[0], l0); atomicMax(&lrange[1], l1 - 1); }
    __syncthreads();
    const int la = lrange[0], lb = lrange[1];  // block-uniform
    for (int l = la; l <= lb; ++l) {
      const unsigned m = __ballot_sync(0xffffffffu, l >= l0 && l < l1);
      if (lane == 0) wc[l][w] = __popc(m);
    }
    __syncthreads();
    for (int l = la; l <= lb; ++l) {
      const unsigned m = __ballot_sync(0xffffffffu, l >= l0 && l < l1);
      if (l >= l0 && l < l1) {
        int64_t pos = boff[(int64_t)l * gridDim.x + blockIdx.x] + __popc(m & ((1u << lane) - 1u));
        for (int q = 0; q < w; ++q) pos += wc[l][q];
        out[pos] = ((uint64_t)l << 32) | (uint64_t)i;
      }
    }
  }
}

__global__ void k_root(int64_t n, int* start, int* count, int* parent, int* level, int* ix,
                       int* iy, uint64_t* code) {
  start[0] = 0; count[0] = (int)n; parent[0] = -1; level[0] = 0; ix[0] = 0; iy[0] = 0; code[0] = 0;
}

__global__ void k_fill_boxes(const uint64_t* __restrict__ splits, int64_t nsplit,
                             LevelOffsets split_off, LevelOffsets box_off,
                             const uint64_t* __restrict__ k, int64_t n, int depth,
                             int* box_start, int* box_count, int* box_child, int* box_parent,
                             int* box_level, int* box_ix, int* box_iy, uint64_t* box_code) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nsplit) return;
  const uint64_t e = splits[g];
  const int l = (int)(e >> 32);
  const int64_t i = (int64_t)(e & 0xffffffffull);
  const int64_t rank = g - split_off.off[l];
  int64_t own = 0;
  if (l > 0) {
    // parent split node: the last entry of level l-1 starting at or before i
    int64_t lo = split_off.off[l - 1], hi = split_off.off[l];
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if ((int64_t)(splits[mid] & 0xffffffffull) <= i) lo = mid + 1; else hi = mid;
    }
    const int64_t prank = (lo - 1) - split_off.off[l - 1];
    const int dig = (int)((k[i] >> (2 * (depth - l))) & 3ull);
    own = box_off.off[l] + 4 * prank + dig;
  }
  const uint64_t mask = (l == 0) ? ~0ull : ((1ull << (2 * (depth - l))) - 1ull);
  const int64_t end = (l == 0) ? n : upper_bound(k, i + 1, n, k[i] | mask);
  const uint64_t P = (l == 0) ? 0ull : (k[i] >> (2 * (depth - l)));
  const int pix = (int)compact2(P), piy = (int)compact2(P >> 1);
  const int64_t c0 = box_off.off[l + 1] + 4 * rank;
  box_child[own] = (int)c0;
  const int sh = 2 * (depth - l - 1);
  int64_t b[5];
  b[0] = i;
  b[4] = end;
  for (int q = 1; q < 4; ++q) b[q] = lower_bound(k, i, end, ((P << 2) | (uint64_t)q) << sh);
  for (int q = 0; q < 4; ++q) {
    const int64_t c = c0 + q;
    box_start[c] = (int)b[q];
    box_count[c] = (int)(b[q + 1] - b[q]);
    box_parent[c] = (int)own;
    box_level[c] = l + 1;
    box_ix[c] = 2 * pix + (q & 1);
    box_iy[c] = 2 * piy + (q >> 1);
    box_code[c] = (P << 2) | (uint64_t)q;
  }
}

struct TreeView {
  const int* start; const int* count; const int* child; const int* level;
  const int* ix; const int* iy; const uint64_t* code;
  LevelOffsets lo;
};

__global__ void k_active_flags(TreeView T, int64_t nb, double root_lo_x, double root_lo_y,
                               double root_size, int has_target, double t0, double t1,
                               double t2, double t3, uint8_t* __restrict__ active,
                               int64_t* __restrict__ fa, int64_t* __restrict__ fl) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  bool act = true;
  if (has_target) {
    const double side = root_size / (double)(1ull << T.level[b]);
    const double x0 = root_lo_x + T.ix[b] * side, y0 = root_lo_y + T.iy[b] * side;
    // a sliver of slack so that rays on the target's edge, whatever rounding
    // produced them, always fall in an active leaf
    const double eps = 1e-9 * root_size;
    act = (x0 <= t1 + eps) && (x0 + side >= t0 - eps) && (y0 <= t3 + eps) && (y0 + side >= t2 - eps);
  }
  active[b] = act ? 1 : 0;
  fa[b] = act ? 1 : 0;
  fl[b] = (act && T.child[b] < 0) ? 1 : 0;
}

__global__ void k_compact(const int64_t* __restrict__ flag, const int64_t* __restrict__ pos,
                          int64_t n, int* __restrict__ out, int* __restrict__ inv) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= n) return;
  if (flag[b]) out[pos[b]] = (int)b;
  if (inv) inv[b] = flag[b] ? (int)pos[b] : -1;
}

// box containing cell (level, ix, iy): the box at that level if it exists,
// else the coarser leaf that covers it; -1 outside the root.
__device__ int find_box(const TreeView& T, int level, long long ix, long long iy) {
  const long long lim = 1ll << level;
  if (ix < 0 || iy < 0 || ix >= lim || iy >= lim) return -1;
  for (int l = level; l >= 0; --l) {
    const uint64_t c = morton((uint32_t)ix, (uint32_t)iy);
    int64_t lo = T.lo.off[l], hi = T.lo.off[l + 1];
    const int64_t end = hi;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (T.code[mid] < c) lo = mid + 1; else hi = mid;
    }
    if (lo < end && T.code[lo] == c) return (int)lo;
    ix >>= 1; iy >>= 1;
  }
  return -1;
}

__device__ __forceinline__ bool adjacent(const TreeView& T, int a, int b) {
  const int la = T.level[a], lb = T.level[b];
  const int L = la > lb ? la : lb;
  const long long ax0 = (long long)T.ix[a] << (L - la), ax1 = (long long)(T.ix[a] + 1) << (L - la);
  const long long ay0 = (long long)T.iy[a] << (L - la), ay1 = (long long)(T.iy[a] + 1) << (L - la);
  const long long bx0 = (long long)T.ix[b] << (L - lb), bx1 = (long long)(T.ix[b] + 1) << (L - lb);
  const long long by0 = (long long)T.iy[b] << (L - lb), by1 = (long long)(T.iy[b] + 1) << (L - lb);
  return ax0 <= bx1 && bx0 <= ax1 && ay0 <= by1 && by0 <= ay1;
}

struct ListOut {
  int64_t* cV; int64_t* cX; int64_t* cU; int64_t* cW;        // counts (pass 1)
  const int64_t* oV; const int64_t* oX; const int64_t* oU; const int64_t* oW;  // offsets (pass 2)
  int* V; int* X; int* U; int* W;
  int64_t* ustars;  // per active index: stars in U (pass 1)
  const int* nbr;   // per active index: 18 neighbour boxes (k_neighbours)
};

// The 18 neighbour lookups of each active box, one thread each: [0..8] the
// boxes at level l-1 around its parent (V and X lists, levels >= 2), [9..17]
// the boxes at level l around it (U and W lists, leaves), in the row-major
// (dy, dx) order the list kernel walks them; -1 outside the root or unused.
// A lookup is a binary search per level, so spreading them over threads
// shortens the chains of dependent loads the list kernel would wait on.
__global__ void k_neighbours(TreeView T, const int* __restrict__ active, int64_t nact,
                             int* __restrict__ nbr) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nact * 18) return;
  const int64_t a = t / 18;
  const int q = (int)(t - a * 18), q9 = q % 9;
  const int dx = q9 % 3 - 1, dy = q9 / 3 - 1;
  const int B = active[a];
  const int l = T.level[B];
  const long long bx = T.ix[B], by = T.iy[B];
  int r = -1;
  if (q < 9) {
    if (l >= 2) r = find_box(T, l - 1, (bx >> 1) + dx, (by >> 1) + dy);
  } else if (T.child[B] < 0) {
    r = find_box(T, l, bx + dx, by + dy);
  }
  nbr[t] = r;
}

template <bool WRITE>
__global__ void k_lists(TreeView T, const int* __restrict__ active, int64_t nact, ListOut o) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nact) return;
  const int B = active[a];
  const int l = T.level[B];
  int64_t nV = 0, nX = 0, nU = 0, nW = 0, us = 0;
  int64_t pV = WRITE ? o.oV[a] : 0, pX = WRITE ? o.oX[a] : 0;
  int64_t pU = WRITE ? o.oU[a] : 0, pW = WRITE ? o.oW[a] : 0;
  if (l >= 2) {
    int seen[9];
    int nseen = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int Q = o.nbr[a * 18 + (dy + 1) * 3 + (dx + 1)];
        if (Q < 0) continue;
        if (T.level[Q] == l - 1 && T.child[Q] >= 0) {
          for (int q = 0; q < 4; ++q) {
            const int C = T.child[Q] + q;
            if (T.count[C] == 0 || adjacent(T, C, B)) continue;
            if (WRITE) o.V[pV++] = C;
            ++nV;
          }
        } else {
          bool dup = false;
          for (int s = 0; s < nseen; ++s) dup |= (seen[s] == Q);
          if (dup) continue;
          seen[nseen++] = Q;
          if (T.count[Q] == 0 || adjacent(T, Q, B)) continue;
          if (WRITE) o.X[pX++] = Q;
          ++nX;
        }
      }
  }
  if (T.child[B] < 0) {
    int seen[9];
    int nseen = 0;
    int stack[128];
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int C = o.nbr[a * 18 + 9 + (dy + 1) * 3 + (dx + 1)];
        if (C < 0) continue;
        if (T.level[C] < l) {
          bool dup = false;
          for (int s = 0; s < nseen; ++s) dup |= (seen[s] == C);
          if (dup) continue;
          seen[nseen++] = C;
          if (T.count[C] > 0) { if (WRITE) o.U[pU++] = C; ++nU; us += T.count[C]; }
          continue;
        }
        if (T.count[C] == 0) continue;
        if (T.child[C] < 0) { if (WRITE) o.U[pU++] = C; ++nU; us += T.count[C]; continue; }
        int sp = 0;
        for (int q = 3; q >= 0; --q) stack[sp++] = T.child[C] + q;
        while (sp > 0) {
          const int Dn = stack[--sp];
          if (T.count[Dn] == 0) continue;
          if (adjacent(T, Dn, B)) {
            if (T.child[Dn] < 0) { if (WRITE) o.U[pU++] = Dn; ++nU; us += T.count[Dn]; }
            else if (sp + 4 <= 128) { for (int q = 3; q >= 0; --q) stack[sp++] = T.child[Dn] + q; }
          } else {
            if (WRITE) o.W[pW++] = Dn;
            ++nW;
          }
        }
      }
  }
  if (!WRITE) {
    o.cV[a] = nV; o.cX[a] = nX; o.cU[a] = nU; o.cW[a] = nW; o.ustars[a] = us;
  }
}

__global__ void k_sentinels(int64_t* a, int64_t* b, int64_t* c, int64_t* d, int64_t va,
                            int64_t vb, int64_t vc, int64_t vd) {
  if (threadIdx.x == 0) { *a = va; *b = vb; *c = vc; *d = vd; }
}

}  // namespace

void tree_build_boxes(Plan& P, const double* stars, const double* masses, cudaStream_t s) {
  const int64_t n = P.n;
  const int depth = P.depth;
  // ---- 1. bounds + finiteness -------------------------------------------
  const int nbb = (int)std::min<int64_t>(1024, (n + 255) / 256);
  std::vector<double> part(kBoundsParts * (size_t)nbb);
  {
    Scratch dpart(&P.da, sizeof(double) * kBoundsParts * nbb);
    k_bounds<<<nbb, kBoundsThreads, 0, s>>>(stars, masses, n, dpart.as<double>());
    LENS_LAUNCHED("k_bounds");
    // the translation tables are formed on the host while the bounds run
    fmm_tables(P, s);
    LENS_CUDA(cudaMemcpyAsync(part.data(), dpart.p, sizeof(double) * kBoundsParts * nbb,
                              cudaMemcpyDeviceToHost, s));
    LENS_CUDA(cudaStreamSynchronize(s));
  }
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY, bad = 0;
  double mmin = INFINITY, mmax = -INFINITY;
  for (int b = 0; b < nbb; ++b) {
    const double* q = &part[(size_t)kBoundsParts * b];
    xmin = std::min(xmin, q[0]); xmax = std::max(xmax, q[1]);
    ymin = std::min(ymin, q[2]); ymax = std::max(ymax, q[3]);
    bad += q[4];
    mmin = std::min(mmin, q[5]); mmax = std::max(mmax, q[6]);
  }
  if (bad > 0) fail(LENS_EINVAL, "non-finite star position or mass");
  // all stars of one mass (a common microlensing field): the float32 near
  // field then sums 1/|d|^2-weighted offsets and scales by the mass once
  P.equal_mass = mmin == mmax;
  P.mass0 = mmin;
  if (P.has_target) {
    xmin = std::min(xmin, P.target[0]); xmax = std::max(xmax, P.target[1]);
    ymin = std::min(ymin, P.target[2]); ymax = std::max(ymax, P.target[3]);
  }
  double size = std::max(xmax - xmin, ymax - ymin);
  const double mag = std::max({std::fabs(xmin), std::fabs(xmax), std::fabs(ymin), std::fabs(ymax), 1e-300});
  if (!(size > 1e-12 * mag)) size = std::max(1.0, 1e-6 * mag);
  size *= 1.0 + 1e-6;
  P.root_size = size;
  P.root_lo[0] = 0.5 * (xmin + xmax) - 0.5 * size;
  P.root_lo[1] = 0.5 * (ymin + ymax) - 0.5 * size;

  // ---- 2. keys + sort + gather ------------------------------------------
  P.skey = P.dalloc_n<uint64_t>(n);
  P.sidx = P.dalloc_n<uint32_t>(n);
  P.spos = P.dalloc_n<double2>(n);
  P.smass = P.dalloc_n<double>(n);
  const double scale = (double)(1ull << depth) / size;
  k_keys<<<grid_for(n, 256), 256, 0, s>>>(stars, n, P.root_lo[0], P.root_lo[1], scale, depth,
                                           P.skey, P.sidx);
  LENS_LAUNCHED("k_keys");
  // Sort by the top key bits only, down to a level the tree is unlikely to
  // pass (6 levels below the depth of a uniform field of n stars, leaf
  // stars per box); if a box of that level still holds more than leaf stars,
  // the keys are sorted again in full.
  int dcap = 6;
  while (dcap < depth && (double)P.leaf * std::pow(4.0, dcap - 6) < (double)n) ++dcap;
  dcap = std::min(depth, dcap);
  const int lo_bit = (2 * (depth - dcap)) / 8 * 8;
  dcap = depth - lo_bit / 2;  // the levels the sorted bits resolve
  radix_sort_u64(P.skey, P.sidx, n, 2 * depth, P.da, s, lo_bit);

  // ---- 3. split nodes ---------------------------------------------------
  Scratch dcnt(&P.da, sizeof(unsigned long long) * (kMaxDepth + 2) + sizeof(int) * 4);
  unsigned long long* counts = dcnt.as<unsigned long long>();
  int* deep = reinterpret_cast<int*>(counts + kMaxDepth + 2);
  const unsigned nblk = grid_for(n, kSplitThreads);
  Scratch bcnt(&P.da, sizeof(int64_t) * kMaxDepth * (size_t)nblk);
  unsigned long long hc[kMaxDepth + 2];
  int hdeep[4];
  for (;;) {
    LENS_CUDA(cudaMemsetAsync(dcnt.p, 0, dcnt.bytes, s));
    k_splits<false><<<nblk, kSplitThreads, 0, s>>>(P.skey, n, depth, dcap, P.leaf, counts, deep,
                                                   bcnt.as<int64_t>(), nullptr, nullptr);
    LENS_LAUNCHED("k_splits<count>");
    LENS_CUDA(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
    LENS_CUDA(cudaMemcpyAsync(hdeep, deep, sizeof(hdeep), cudaMemcpyDeviceToHost, s));
    LENS_CUDA(cudaStreamSynchronize(s));
    if (!hdeep[0]) break;
    if (dcap == depth)
      fail(LENS_EDEPTH, "a box at the depth cap still holds more than leaf_size stars "
                        "(coincident stars?): raise leaf_size or max_depth");
    // deeper than the partial sort resolves: sort the low bits too (all
    // passes again, least significant first)
    radix_sort_u64(P.skey, P.sidx, n, 2 * depth, P.da, s, 0);
    dcap = depth;
  }
  k_gather<<<grid_for(n, 256), 256, 0, s>>>(stars, masses, P.sidx, n, P.spos, P.smass);
  LENS_LAUNCHED("k_gather");
  LevelOffsets soff{}, boff{};
  int64_t nsplit = 0;
  int maxl = -1;
  for (int l = 0; l < depth; ++l) {
    soff.off[l] = nsplit;
    nsplit += (int64_t)hc[l];
    if (hc[l]) maxl = l;
  }
  for (int l = depth; l <= kMaxDepth + 1; ++l) soff.off[l] = nsplit;
  P.nlevels = maxl + 2;  // levels 0 .. maxl+1
  P.level_off.assign(P.nlevels + 1, 0);
  P.level_off[0] = 0;
  P.level_off[1] = 1;
  for (int l = 1; l < P.nlevels; ++l) P.level_off[l + 1] = P.level_off[l] + 4 * (int64_t)hc[l - 1];
  P.nb = P.level_off[P.nlevels];
  if (P.nb > (int64_t)INT32_MAX) fail(LENS_ENOMEM, "tree too large");
  for (int l = 0; l <= kMaxDepth + 1; ++l)
    boff.off[l] = l <= P.nlevels ? P.level_off[l] : P.nb;
  boff.nlevels = P.nlevels;

  const int64_t nb = P.nb;
  P.box_start = P.dalloc_n<int>(nb);
  P.box_count = P.dalloc_n<int>(nb);
  P.box_child = P.dalloc_n<int>(nb);
  P.box_parent = P.dalloc_n<int>(nb);
  P.box_level = P.dalloc_n<int>(nb);
  P.box_ix = P.dalloc_n<int>(nb);
  P.box_iy = P.dalloc_n<int>(nb);
  P.box_code = P.dalloc_n<uint64_t>(nb);
  P.box_active = P.dalloc_n<uint8_t>(nb);
  LENS_CUDA(cudaMemsetAsync(P.box_child, 0xff, sizeof(int) * nb, s));
  k_root<<<1, 1, 0, s>>>(n, P.box_start, P.box_count, P.box_parent, P.box_level, P.box_ix,
                          P.box_iy, P.box_code);
  LENS_LAUNCHED("k_root");
  if (nsplit > 0) {
    Scratch dspl(&P.da, sizeof(uint64_t) * nsplit);
    Scratch bpos(&P.da, sizeof(int64_t) * kMaxDepth * (size_t)nblk);
    exclusive_scan_i64(bcnt.as<int64_t>(), bpos.as<int64_t>(), (int64_t)kMaxDepth * nblk, P.da, s);
    k_splits<true><<<nblk, kSplitThreads, 0, s>>>(P.skey, n, depth, dcap, P.leaf, nullptr, nullptr,
                                                  nullptr, bpos.as<int64_t>(), dspl.as<uint64_t>());
    LENS_LAUNCHED("k_splits<write>");
    k_fill_boxes<<<grid_for(nsplit, 256), 256, 0, s>>>(
        dspl.as<uint64_t>(), nsplit, soff, boff, P.skey, n, depth, P.box_start, P.box_count,
        P.box_child, P.box_parent, P.box_level, P.box_ix, P.box_iy, P.box_code);
    LENS_LAUNCHED("k_fill_boxes");
  }

}

void tree_build_lists(Plan& P, cudaStream_t s) {
  const int64_t nb = P.nb;
  LevelOffsets boff{};
  for (int l = 0; l <= kMaxDepth + 1; ++l)
    boff.off[l] = l <= P.nlevels ? P.level_off[l] : P.nb;
  boff.nlevels = P.nlevels;
  // ---- 4. active boxes -------------------------------------------------
  TreeView T{P.box_start, P.box_count, P.box_child, P.box_level, P.box_ix, P.box_iy,
             P.box_code, boff};
  Scratch fa(&P.da, sizeof(int64_t) * nb), fl(&P.da, sizeof(int64_t) * nb);
  Scratch pa(&P.da, sizeof(int64_t) * nb), pl(&P.da, sizeof(int64_t) * nb);
  k_active_flags<<<grid_for(nb, 256), 256, 0, s>>>(
      T, nb, P.root_lo[0], P.root_lo[1], P.root_size, P.has_target ? 1 : 0, P.target[0],
      P.target[1], P.target[2], P.target[3], P.box_active, fa.as<int64_t>(), fl.as<int64_t>());
  LENS_LAUNCHED("k_active_flags");
  exclusive_scan_i64(fa.as<int64_t>(), pa.as<int64_t>(), nb, P.da, s);
  exclusive_scan_i64(fl.as<int64_t>(), pl.as<int64_t>(), nb, P.da, s);
  std::vector<int64_t> hpos(P.nlevels + 1);
  int64_t lastf[2], lastp[2];
  {
    // level starts of the active list and the two totals, in one read-back
    std::vector<const int64_t*> addr;
    for (int l = 0; l < P.nlevels; ++l) addr.push_back(pa.as<int64_t>() + P.level_off[l]);
    addr.push_back(fa.as<int64_t>() + nb - 1);
    addr.push_back(pa.as<int64_t>() + nb - 1);
    addr.push_back(fl.as<int64_t>() + nb - 1);
    addr.push_back(pl.as<int64_t>() + nb - 1);
    std::vector<int64_t> v(addr.size());
    read_i64(addr.data(), (int)addr.size(), v.data(), P.da, s);
    for (int l = 0; l < P.nlevels; ++l) hpos[l] = v[l];
    lastf[0] = v[P.nlevels]; lastp[0] = v[P.nlevels + 1];
    lastf[1] = v[P.nlevels + 2]; lastp[1] = v[P.nlevels + 3];
  }
  P.n_active = lastf[0] + lastp[0];
  P.n_active_leaves = lastf[1] + lastp[1];
  hpos[P.nlevels] = P.n_active;
  P.active_level_off = hpos;
  P.active = P.dalloc_n<int>(P.n_active);
  P.active_leaves = P.dalloc_n<int>(P.n_active_leaves);
  P.box_aidx = P.dalloc_n<int>(nb);
  k_compact<<<grid_for(nb, 256), 256, 0, s>>>(fa.as<int64_t>(), pa.as<int64_t>(), nb, P.active,
                                               P.box_aidx);
  LENS_LAUNCHED("k_compact");
  P.box_lidx = P.dalloc_n<int>(nb);
  k_compact<<<grid_for(nb, 256), 256, 0, s>>>(fl.as<int64_t>(), pl.as<int64_t>(), nb,
                                               P.active_leaves, P.box_lidx);
  LENS_LAUNCHED("k_compact");

  // ---- 5. interaction lists ------------------------------------------
  const int64_t na = P.n_active;
  Scratch cnt(&P.da, sizeof(int64_t) * 5 * (na + 1));
  int64_t* c = cnt.as<int64_t>();
  ListOut o{};
  o.cV = c; o.cX = c + na; o.cU = c + 2 * na; o.cW = c + 3 * na; o.ustars = c + 4 * na;
  Scratch nbr(&P.da, sizeof(int) * 18 * (size_t)std::max<int64_t>(na, 1));
  if (na > 0) {
    k_neighbours<<<grid_for(na * 18, 256), 256, 0, s>>>(T, P.active, na, nbr.as<int>());
    LENS_LAUNCHED("k_neighbours");
  }
  o.nbr = nbr.as<int>();
  k_lists<false><<<grid_for(na, 128), 128, 0, s>>>(T, P.active, na, o);
  LENS_LAUNCHED("k_lists<count>");
  int64_t* offs[4];
  int64_t tot[4];
  for (int q = 0; q < 4; ++q) {
    offs[q] = reinterpret_cast<int64_t*>(P.dalloc(sizeof(int64_t) * (na + 1)));
    exclusive_scan_i64(c + q * na, offs[q], na, P.da, s);
  }
  // totals: last offset + last count; also total U stars
  std::vector<int64_t> hl(10, 0);
  P.ustar_cnt = P.dalloc_n<int64_t>(na + 1);
  if (na > 0)
    LENS_CUDA(cudaMemcpyAsync(P.ustar_cnt, c + 4 * na, sizeof(int64_t) * na,
                              cudaMemcpyDeviceToDevice, s));
  Scratch usum(&P.da, sizeof(int64_t) * (na + 1));
  if (na > 0) {
    exclusive_scan_i64(c + 4 * na, usum.as<int64_t>(), na, P.da, s);
    const int64_t* addr[10];
    for (int q = 0; q < 4; ++q) {
      addr[2 * q] = offs[q] + na - 1;
      addr[2 * q + 1] = c + q * na + na - 1;
    }
    addr[8] = usum.as<int64_t>() + na - 1;
    addr[9] = c + 4 * na + na - 1;
    read_i64(addr, 10, hl.data(), P.da, s);
  }
  for (int q = 0; q < 4; ++q) tot[q] = hl[2 * q] + hl[2 * q + 1];
  P.u_stars = hl[8] + hl[9];
  // write the totals as the sentinel offsets[na] (kernel parameters: no host
  // buffer has to outlive the call)
  k_sentinels<<<1, 32, 0, s>>>(offs[0] + na, offs[1] + na, offs[2] + na, offs[3] + na, tot[0],
                               tot[1], tot[2], tot[3]);
  LENS_LAUNCHED("k_sentinels");
  P.nV = tot[0]; P.nX = tot[1]; P.nU = tot[2]; P.nW = tot[3];
  P.V_list = P.dalloc_n<int>(tot[0]);
  P.X_list = P.dalloc_n<int>(tot[1]);
  P.U_list = P.dalloc_n<int>(tot[2]);
  P.W_list = P.dalloc_n<int>(tot[3]);
  o.oV = offs[0]; o.oX = offs[1]; o.oU = offs[2]; o.oW = offs[3];
  o.V = P.V_list; o.X = P.X_list; o.U = P.U_list; o.W = P.W_list;
  k_lists<true><<<grid_for(na, 128), 128, 0, s>>>(T, P.active, na, o);
  LENS_LAUNCHED("k_lists<write>");
  P.V_off = offs[0];
  P.X_off = offs[1];
  P.U_off = offs[2];
  P.W_off = offs[3];
}

}  // namespace lens
