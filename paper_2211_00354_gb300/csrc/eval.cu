// eval.cu -- the per-ray FMM evaluation, fused: L2P (Appendix A, step 6),
// P2P with the adjacent leaves (step 7), M2P for the adaptive W lists, and
// the lens equation y = diag(1-kappa_s-gamma, 1-kappa_s+gamma) x - alpha
// (Eq. 1 with the smooth field) with an optional Jacobian dy/dx.
//
// One CTA works on one tile of rays that lie in one active leaf B.  The stars
// of B's U list are staged in shared memory as offsets from B's centre (formed
// in float64 once per CTA, then rounded), so in the float32 form a near-field
// difference d = (x - c) - (x_j - c) keeps float32 relative accuracy even
// far from the origin.  Each U leaf's contribution is summed in plain float32
// and added to a two-sum (hi, lo) accumulator (compensated per source leaf).
// The local expansion is evaluated by Horner in w = (x - c)/r with b_0 kept
// in float64.  y is formed in float64.
//
// Grid path: the rays of a leaf are an index rectangle of the image-plane
// grid (x = x0 + i h), so no ray array exists; a ray belongs to the leaf whose
// half-open box [lo, hi) holds it.  Ray path: rays are bucketed by leaf first.
#include <algorithm>
#include <vector>

#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kEvalThreads = 128;
constexpr int kSeg = 64;    // U entries staged per round
constexpr int kChunk = 1024; // stars staged per sub-round
constexpr int kWChunk = 8;  // W entries staged per round

struct EvalArgs {
  const double2* spos; const double* smass;
  const int* start; const int* count; const int* level; const int* ix; const int* iy;
  const int* aidx;
  const int64_t* U_off; const int* U_list; const int64_t* W_off; const int* W_list;
  const double2* M; const double2* L;
  const int* leaves;
  const int2* tile_leaf;  // (leaf, tile within the leaf) of each block
  int64_t nleaf;
  double lo_x, lo_y, root_size;
  int p;
  double a, b;
  // grid source
  const int64_t* rect;  // per leaf: i0, ni, j0, nj
  double gx0, gy0, gh;
  int64_t gnx1, grow0;
  // ray source
  const double* rays; const int64_t* ray_off; const int* perm;
  double* y; double* jac;
  // pixel-coordinate output (IPM path): u = y1 * pinv_du + pu_off, etc.
  PixCorner* pix;
  double pinv_du, pu_off, pinv_dv, pv_off;
};

__device__ __forceinline__ double grid_coord(double x0, int64_t i, double h) {
  return __dadd_rn(x0, __dmul_rn((double)i, h));
}

// The float64 form of the fused evaluation (the float32-bulk form is
// eval32.cu): one CTA per (leaf, tile of rays), the leaf's U-list stars
// staged in shared memory in rounds, M2P for the W list, L2P by Horner, and
// the lens equation y = diag(a, b) x - alpha in float64.
template <bool JAC, bool GRID, bool PIX, int RPT>
__global__ void __launch_bounds__(kEvalThreads) k_eval(EvalArgs A) {
  __shared__ double s_x[kChunk], s_y[kChunk], s_m[kChunk];
  __shared__ int s_pre[kSeg + 1];
  __shared__ int s_box[kSeg];
  __shared__ double2 s_L[kMaxOrder + 1];
  __shared__ double2 s_W[kWChunk][kMaxOrder + 1];
  __shared__ double s_wx[kWChunk], s_wy[kWChunk], s_wr[kWChunk];
  const int tid = threadIdx.x;
  const int p = A.p;
  const int2 kt = A.tile_leaf[blockIdx.x];
  const int64_t k = kt.x;
  const int B = A.leaves[k];
  const int a = A.aidx[B];
  const int64_t tile = kt.y;
  const int lv = A.level[B];
  const double r = A.root_size / (double)(2ull << lv);
  const double cx = A.lo_x + (2.0 * A.ix[B] + 1.0) * r;
  const double cy = A.lo_y + (2.0 * A.iy[B] + 1.0) * r;
  const double2* Lb = A.L + (int64_t)B * (p + 1);
  for (int l = tid; l <= p; l += kEvalThreads) s_L[l] = Lb[l];
  // rays of this tile
  int64_t nr_leaf, i0 = 0, ni = 1, j0 = 0;
  if (GRID) {
    i0 = A.rect[4 * k]; ni = A.rect[4 * k + 1]; j0 = A.rect[4 * k + 2];
    nr_leaf = ni * A.rect[4 * k + 3];
  } else {
    nr_leaf = A.ray_off[k + 1] - A.ray_off[k];
  }
  double dx[RPT], dy[RPT], x1[RPT], x2[RPT];
  int64_t oidx[RPT];
  bool ok[RPT];
  double n1[RPT], n2[RPT], nj1[RPT], nj2[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int64_t loc = tile * (kEvalThreads * RPT) + (int64_t)q * kEvalThreads + tid;
    ok[q] = loc < nr_leaf;
    x1[q] = cx; x2[q] = cy; oidx[q] = 0;
    if (ok[q]) {
      if (GRID) {
        // 32-bit division: a 64-bit one is emulated with float64 instructions
        const uint32_t l32 = (uint32_t)loc, n32 = (uint32_t)ni;
        const uint32_t dj32 = l32 / n32;
        const int64_t dj = dj32, di = (int64_t)(l32 - dj32 * n32);
        const int64_t i = i0 + di, j = j0 + dj;
        oidx[q] = (j - A.grow0) * A.gnx1 + i;
        x1[q] = grid_coord(A.gx0, i, A.gh);
        x2[q] = grid_coord(A.gy0, j, A.gh);
      } else {
        const int64_t ridx = A.perm[A.ray_off[k] + loc];
        x1[q] = A.rays[2 * ridx];
        x2[q] = A.rays[2 * ridx + 1];
        oidx[q] = ridx;
      }
    }
    dx[q] = x1[q] - cx;
    dy[q] = x2[q] - cy;
    n1[q] = 0.0; n2[q] = 0.0; nj1[q] = 0.0; nj2[q] = 0.0;
  }
  // ---- P2P over the U list ----------------------------------------------
  const int64_t u_beg = A.U_off[a], u_end = A.U_off[a + 1];
  for (int64_t e0 = u_beg; e0 < u_end; e0 += kSeg) {
    const int ne = (int)min64(kSeg, u_end - e0);
    __syncthreads();
    if (tid < 32) {
      int base = 0;
      for (int half = 0; half < kSeg / 32; ++half) {
        const int e = half * 32 + tid;
        int box = -1, c = 0;
        if (e < ne) { box = A.U_list[e0 + e]; c = A.count[box]; }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (tid >= o) incl += v;
        }
        if (e < kSeg) { s_box[e] = box; s_pre[e + 1] = base + incl; }
        base += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (tid == 0) s_pre[0] = 0;
    }
    __syncthreads();
    const int tot = s_pre[ne];
    for (int f0 = 0; f0 < tot; f0 += kChunk) {
      const int nf = min(kChunk, tot - f0);
      if (f0 > 0) __syncthreads();
      for (int f = tid; f < nf; f += kEvalThreads) {
        const int ff = f0 + f;
        int lo = 0, hi = ne;  // entry e with s_pre[e] <= ff < s_pre[e+1]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_pre[mid] <= ff) lo = mid; else hi = mid;
        }
        const int st = A.start[s_box[lo]] + (ff - s_pre[lo]);
        const double2 z = A.spos[st];
        s_x[f] = z.x - cx;
        s_y[f] = z.y - cy;
        s_m[f] = A.smass[st];
      }
      __syncthreads();
      for (int e = 0; e < ne; ++e) {
        const int lo = max(s_pre[e], f0) - f0;
        const int hi = min(s_pre[e + 1], f0 + nf) - f0;
        if (hi <= lo) continue;
        double p1[RPT], p2[RPT], pj1[RPT], pj2[RPT];
#pragma unroll
        for (int q = 0; q < RPT; ++q) { p1[q] = 0; p2[q] = 0; pj1[q] = 0; pj2[q] = 0; }
        for (int j = lo; j < hi; ++j) {
          const double sx = s_x[j], sy = s_y[j], sm = s_m[j];
#pragma unroll
          for (int q = 0; q < RPT; ++q) {
            const double d1 = dx[q] - sx, d2 = dy[q] - sy;
            const double r2 = d1 * d1 + d2 * d2;
            // a star exactly on the ray contributes nothing
            const double inv = r2 > 0.0 ? 1.0 / r2 : 0.0;
            const double w = sm * inv;
            p1[q] += w * d1;
            p2[q] += w * d2;
            if (JAC) {
              const double w2 = w * inv;
              pj1[q] += w2 * (d2 - d1) * (d2 + d1);  // Re f'
              pj2[q] += w2 * (2.0 * d1 * d2);        // Im f'
            }
          }
        }
        // per-source-leaf partial sums
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          n1[q] += p1[q]; n2[q] += p2[q];
          if (JAC) { nj1[q] += pj1[q]; nj2[q] += pj2[q]; }
        }
      }
    }
  }
  // ---- M2P over the W list ----------------------------------------------
  double2 fw[RPT], dfw[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) { fw[q] = make_double2(0, 0); dfw[q] = make_double2(0, 0); }
  const int64_t w_beg = A.W_off[a], w_end = A.W_off[a + 1];
  for (int64_t e0 = w_beg; e0 < w_end; e0 += kWChunk) {
    const int nw = (int)min64(kWChunk, w_end - e0);
    __syncthreads();
    for (int t = tid; t < nw * (p + 1); t += kEvalThreads) {
      const int w = t / (p + 1), kk = t - w * (p + 1);
      s_W[w][kk] = A.M[(int64_t)A.W_list[e0 + w] * (p + 1) + kk];
    }
    if (tid < nw) {
      const int Wb = A.W_list[e0 + tid];
      const double rw = A.root_size / (double)(2ull << A.level[Wb]);
      s_wx[tid] = A.lo_x + (2.0 * A.ix[Wb] + 1.0) * rw - cx;
      s_wy[tid] = A.lo_y + (2.0 * A.iy[Wb] + 1.0) * rw - cy;
      s_wr[tid] = rw;
    }
    __syncthreads();
    for (int w = 0; w < nw; ++w) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const double2 z = make_double2(dx[q] - s_wx[w], dy[q] - s_wy[w]);
        const double2 inv = cinv(z);
        const double2 qq = make_double2(inv.x * s_wr[w], inv.y * s_wr[w]);
        double2 s = s_W[w][p];
        for (int kk = p - 1; kk >= 0; --kk) s = cfma(s, qq, s_W[w][kk]);
        fw[q] = cfma(s, inv, fw[q]);
        if (JAC) {
          double2 t = make_double2((double)(p + 1) * s_W[w][p].x, (double)(p + 1) * s_W[w][p].y);
          for (int kk = p - 1; kk >= 0; --kk)
            t = cfma(t, qq, make_double2((double)(kk + 1) * s_W[w][kk].x, (double)(kk + 1) * s_W[w][kk].y));
          const double2 d = cmul(t, cmul(inv, inv));
          dfw[q] = make_double2(dfw[q].x - d.x, dfw[q].y - d.y);
        }
      }
    }
  }
  // ---- L2P + lens equation ------------------------------------------------
  // alpha = conj(f_total), f_total = b0 + f + near:
  // y1 = a x1 - (Re b0 + Re f + near_1), y2 = b x2 - (-Im b0 - Im f + near_2)
  __syncthreads();
  const double ir = 1.0 / r;
  const double2 b0 = Lb[0];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    if (!ok[q]) continue;
    const double2 w = make_double2(dx[q] * ir, dy[q] * ir);
    double2 f = make_double2(0, 0), df = make_double2(0, 0);
    if (p >= 1) {
      double2 s = s_L[p];
      for (int l = p - 1; l >= 1; --l) s = cfma(s, w, s_L[l]);
      f = cmul(s, w);
      if (JAC) {
        double2 t = make_double2((double)p * s_L[p].x, (double)p * s_L[p].y);
        for (int l = p - 1; l >= 1; --l) t = cfma(t, w, make_double2((double)l * s_L[l].x, (double)l * s_L[l].y));
        df = make_double2(t.x * ir, t.y * ir);
      }
    }
    f = f + fw[q];
    const double al1 = b0.x + f.x + n1[q];
    const double al2 = -(b0.y + f.y) + n2[q];
    const double y1 = fma(A.a, x1[q], -al1);
    const double y2 = fma(A.b, x2[q], -al2);
    if (PIX) {
      const double u = fma(y1, A.pinv_du, A.pu_off), v = fma(y2, A.pinv_dv, A.pv_off);
      PixCorner pc;
      if (fabs(u) < 1073741824.0 && fabs(v) < 1073741824.0) {
        const double fu = floor(u), fv = floor(v);
        pc.iu = (int)fu; pc.fu = (float)(u - fu);
        pc.iv = (int)fv; pc.fv = (float)(v - fv);
      } else {
        pc.iu = 0x7fffffff; pc.fu = 0.f; pc.iv = 0x7fffffff; pc.fv = 0.f;
      }
      A.pix[oidx[q]] = pc;
      continue;
    }
    A.y[2 * oidx[q]] = y1;
    A.y[2 * oidx[q] + 1] = y2;
    if (JAC) {
      const double dre = df.x + dfw[q].x + nj1[q];
      const double dim = df.y + dfw[q].y + nj2[q];
      A.jac[4 * oidx[q] + 0] = A.a - dre;
      A.jac[4 * oidx[q] + 1] = dim;
      A.jac[4 * oidx[q] + 2] = dim;
      A.jac[4 * oidx[q] + 3] = A.b + dre;
    }
  }
}

constexpr int kRptD = 2;

__device__ __forceinline__ int64_t first_at_or_above(double x0, double h, int64_t lo, int64_t hi,
                                                     double bound) {
  // smallest i in [lo, hi] with x0 + i h >= bound (hi if none)
  double g = ceil((bound - x0) / h);
  int64_t i = g < (double)lo ? lo : (g > (double)hi ? hi : (int64_t)g);
  while (i > lo && grid_coord(x0, i - 1, h) >= bound) --i;
  while (i < hi && grid_coord(x0, i, h) < bound) ++i;
  return i;
}

__global__ void k_grid_rects(const int* __restrict__ leaves, int64_t nleaf,
                             const int* __restrict__ level, const int* __restrict__ ix,
                             const int* __restrict__ iy, double lo_x, double lo_y, double size,
                             double x0, double y0, double h, int64_t nx, int64_t row0,
                             int64_t nrows, int tile, int64_t* __restrict__ rect,
                             int64_t* __restrict__ tiles) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nleaf) return;
  const int B = leaves[k];
  const double side = size / (double)(1ull << level[B]);
  const double bx0 = lo_x + ix[B] * side, bx1 = lo_x + (ix[B] + 1) * side;
  const double by0 = lo_y + iy[B] * side, by1 = lo_y + (iy[B] + 1) * side;
  const int64_t i0 = first_at_or_above(x0, h, 0, nx + 1, bx0);
  const int64_t i1 = first_at_or_above(x0, h, 0, nx + 1, bx1);
  const int64_t j0 = first_at_or_above(y0, h, row0, row0 + nrows, by0);
  const int64_t j1 = first_at_or_above(y0, h, row0, row0 + nrows, by1);
  const int64_t ni = i1 > i0 ? i1 - i0 : 0, nj = j1 > j0 ? j1 - j0 : 0;
  rect[4 * k] = i0; rect[4 * k + 1] = ni; rect[4 * k + 2] = j0; rect[4 * k + 3] = nj;
  tiles[k] = (ni * nj + tile - 1) / tile;
}

// algorithmic work of one grid band: rays, ray-star pairs, ray-box M2P evals.
// FP64 form: near stars and W boxes per active box (ustar, W_off); FP32 form
// (near_by_leaf != null): per active leaf, after small W boxes moved to P2P.
__global__ void k_work_count(const int* __restrict__ leaves, int64_t nleaf,
                             const int* __restrict__ aidx, const int64_t* __restrict__ rect,
                             const int64_t* __restrict__ ustar, const int64_t* __restrict__ W_off,
                             const int64_t* __restrict__ near_by_leaf,
                             const int64_t* __restrict__ far_by_leaf, double* __restrict__ work) {
  __shared__ double sh[3][128];
  double r = 0, pp = 0, mw = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nleaf;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double nr = (double)rect[4 * k + 1] * (double)rect[4 * k + 3];
    r += nr;
    if (near_by_leaf) {
      pp += nr * (double)near_by_leaf[k];
      mw += nr * (double)far_by_leaf[k];
    } else {
      const int a = aidx[leaves[k]];
      pp += nr * (double)ustar[a];
      mw += nr * (double)(W_off[a + 1] - W_off[a]);
    }
  }
  sh[0][threadIdx.x] = r; sh[1][threadIdx.x] = pp; sh[2][threadIdx.x] = mw;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) atomicAdd(&work[threadIdx.x], sh[threadIdx.x][0]);
}

__global__ void k_ray_leaf(const double* __restrict__ rays, int64_t m, const int* __restrict__ child,
                           const int* __restrict__ lidx, double lo_x, double lo_y, double scale,
                           int depth, int* __restrict__ slot, int64_t* __restrict__ counts,
                           int* __restrict__ err) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const double x = rays[2 * r], y = rays[2 * r + 1];
  const double qmax = (double)((1u << depth) - 1u);
  const double fx = floor((x - lo_x) * scale), fy = floor((y - lo_y) * scale);
  if (!(fx >= 0.0 && fx <= qmax && fy >= 0.0 && fy <= qmax)) {  // also catches NaN
    atomicExch(err, 1);
    slot[r] = -1;
    return;
  }
  const uint32_t qx = (uint32_t)fx, qy = (uint32_t)fy;
  int b = 0;
  for (int l = 0; l < depth; ++l) {
    const int c = child[b];
    if (c < 0) break;
    const int sh = depth - l - 1;
    b = c + (int)(((qx >> sh) & 1u) | (((qy >> sh) & 1u) << 1));
  }
  const int li = lidx[b];
  if (li < 0) {
    atomicExch(err, 1);
    slot[r] = -1;
    return;
  }
  slot[r] = li;
  // rays of a warp mostly share a leaf (grid rays, sorted rays): one atomic
  // per group of lanes with the same leaf
  const unsigned grp = __match_any_sync(__activemask(), li);
  if ((threadIdx.x & 31) == __ffs(grp) - 1)
    atomicAdd((unsigned long long*)&counts[li], (unsigned long long)__popc(grp));
}

__global__ void k_ray_scatter(const int* __restrict__ slot, int64_t m, const int64_t* __restrict__ off,
                              int64_t* __restrict__ cursor, int* __restrict__ perm) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int li = slot[r];
  if (li < 0) return;
  // one cursor fetch per group of lanes with the same leaf; each lane takes
  // the place of its rank in the group
  const unsigned grp = __match_any_sync(__activemask(), li);
  const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd((unsigned long long*)&cursor[li], (unsigned long long)__popc(grp));
  base = __shfl_sync(grp, base, leader);
  perm[off[li] + (int64_t)base + __popc(grp & ((1u << lane) - 1u))] = (int)r;
}

__global__ void k_tiles_from_counts(const int64_t* __restrict__ counts, int64_t n, int tile,
                                    int64_t* __restrict__ tiles) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  tiles[k] = (counts[k] + tile - 1) / tile;
}

// (leaf, tile within the leaf) of every ray tile, one thread per tile, so
// that each block of the evaluation kernels finds its leaf with one load.
// The offsets are an exclusive scan (toff[0] = 0, toff[nl] = total): the
// tile's leaf is the last one whose offset is at or below it, found by
// bisection with toff[lo] <= t < toff[hi] held throughout; a leaf of no
// tiles shares its offset with the next and is passed over.
__global__ void k_tile_leaf(const int64_t* __restrict__ toff, int64_t nl, int64_t total,
                            int2* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  int64_t lo = 0, hi = nl;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (toff[mid] <= t) lo = mid; else hi = mid;
  }
  out[t] = make_int2((int)lo, (int)(t - toff[lo]));
}

Scratch tile_leaves(Plan& P, const int64_t* toff, int64_t nl, int64_t total, cudaStream_t s) {
  if (total > (int64_t)INT32_MAX) fail(LENS_EINVAL, "too many ray tiles in one call");
  Scratch tl(&P.da, sizeof(int2) * (size_t)std::max<int64_t>(total, 1));
  k_tile_leaf<<<grid_for(total, 256), 256, 0, s>>>(toff, nl, total, tl.as<int2>());
  LENS_LAUNCHED("k_tile_leaf");
  return tl;
}

template <bool GRID, bool PIX>
void launch_eval(Plan& P, EvalArgs& A, int64_t total_tiles, bool jac, cudaStream_t s) {
  if (total_tiles <= 0) return;
  if (total_tiles > (int64_t)INT32_MAX) fail(LENS_EINVAL, "too many ray tiles in one call");
  const unsigned g = (unsigned)total_tiles;
  // float64 form only; the float32-bulk form runs k_eval32 (eval32.cu)
  if (jac) k_eval<true, GRID, PIX, kRptD><<<g, kEvalThreads, 0, s>>>(A);
  else k_eval<false, GRID, PIX, kRptD><<<g, kEvalThreads, 0, s>>>(A);
  LENS_LAUNCHED("k_eval");
}

EvalArgs base_args(Plan& P) {
  EvalArgs A{};
  A.spos = P.spos; A.smass = P.smass;
  A.start = P.box_start; A.count = P.box_count; A.level = P.box_level;
  A.ix = P.box_ix; A.iy = P.box_iy; A.aidx = P.box_aidx;
  A.U_off = P.U_off; A.U_list = P.U_list; A.W_off = P.W_off; A.W_list = P.W_list;
  A.M = P.M; A.L = P.L;
  A.leaves = P.active_leaves;
  A.nleaf = P.n_active_leaves;
  A.lo_x = P.root_lo[0]; A.lo_y = P.root_lo[1]; A.root_size = P.root_size;
  A.p = P.p;
  A.a = 1.0 - P.kappa_s - P.gamma;
  A.b = 1.0 - P.kappa_s + P.gamma;
  return A;
}

int tile_rays(const Plan& P) {
  return P.prec == LENS_FP64 ? kEvalThreads * kRptD : kEval32Threads * kEval32Rpt;
}

}  // namespace

namespace {
template <bool PIX>
void grid_impl(Plan& P, const GridRows& g, double* y, double* jac, PixCorner* pix,
               const IpmParams* ip, cudaStream_t s) {
  const int64_t nl = P.n_active_leaves;
  if (nl == 0 || g.nrows <= 0) return;
  const int tile = tile_rays(P);
  Scratch rect(&P.da, sizeof(int64_t) * 4 * nl);
  Scratch tiles(&P.da, sizeof(int64_t) * (nl + 1));
  Scratch toff(&P.da, sizeof(int64_t) * (nl + 1));
  k_grid_rects<<<grid_for(nl, 128), 128, 0, s>>>(P.active_leaves, nl, P.box_level, P.box_ix,
                                                 P.box_iy, P.root_lo[0], P.root_lo[1],
                                                 P.root_size, g.x0, g.y0, g.h, g.nx, g.row0,
                                                 g.nrows, tile, rect.as<int64_t>(),
                                                 tiles.as<int64_t>());
  LENS_LAUNCHED("k_grid_rects");
  LENS_CUDA(cudaMemsetAsync(tiles.as<int64_t>() + nl, 0, sizeof(int64_t), s));
  exclusive_scan_i64(tiles.as<int64_t>(), toff.as<int64_t>(), nl + 1, P.da, s);
  int64_t total = 0;
  LENS_CUDA(cudaMemcpyAsync(&total, toff.as<int64_t>() + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaStreamSynchronize(s));
  if (P.work) {
    k_work_count<<<grid_for(nl, 128, 1024), 128, 0, s>>>(P.active_leaves, nl, P.box_aidx,
                                                        rect.as<int64_t>(), P.ustar_cnt,
                                                        P.W_off, P.f_ncnt, P.f_wcnt, P.work);
    LENS_LAUNCHED("k_work_count");
  }
  Scratch tl = tile_leaves(P, toff.as<int64_t>(), nl, total, s);
  if (P.prec == LENS_FP32_BULK) {
    eval32_grid(P, g, rect.as<int64_t>(), tl.as<int2>(), total, y, jac, pix, ip, s);
    return;
  }
  wait_expansions(P, s);
  EvalArgs A = base_args(P);
  A.tile_leaf = tl.as<int2>();
  A.rect = rect.as<int64_t>();
  A.gx0 = g.x0; A.gy0 = g.y0; A.gh = g.h;
  A.gnx1 = g.nx + 1; A.grow0 = g.row0;
  A.y = y; A.jac = jac; A.pix = pix;
  if (PIX) {
    A.pinv_du = ip->inv_du; A.pu_off = -ip->u0 * ip->inv_du;
    A.pinv_dv = ip->inv_dv; A.pv_off = -ip->v0 * ip->inv_dv;
  }
  if (P.timing) {
    auto e = event_pair_begin(s);
    launch_eval<true, PIX>(P, A, total, jac != nullptr, s);
    event_pair_end(e, s);
    P.ev_eval.push_back(e);
  } else {
    launch_eval<true, PIX>(P, A, total, jac != nullptr, s);
  }
}
}  // namespace

void evaluate_grid_fused(Plan& P, const GridRows& g, PixCorner* edge, const IpmParams& ip,
                         float* map32, float* rowdiff, double* stats_dev, int* queue, int* qcount,
                         int* rq, int* rqcount, cudaStream_t s) {
  const int64_t nl = P.n_active_leaves;
  if (nl == 0 || g.nrows <= 0) return;
  if (P.prec != LENS_FP32_BULK) fail(LENS_EINVAL, "the fused map path needs a float32-bulk plan");
  Scratch rect(&P.da, sizeof(int64_t) * 4 * nl);
  Scratch tiles(&P.da, sizeof(int64_t) * (nl + 1));
  k_grid_rects<<<grid_for(nl, 128), 128, 0, s>>>(P.active_leaves, nl, P.box_level, P.box_ix,
                                                 P.box_iy, P.root_lo[0], P.root_lo[1],
                                                 P.root_size, g.x0, g.y0, g.h, g.nx, g.row0,
                                                 g.nrows, tile_rays(P), rect.as<int64_t>(),
                                                 tiles.as<int64_t>());
  LENS_LAUNCHED("k_grid_rects");
  if (P.work) {
    k_work_count<<<grid_for(nl, 128, 1024), 128, 0, s>>>(P.active_leaves, nl, P.box_aidx,
                                                        rect.as<int64_t>(), P.ustar_cnt,
                                                        P.W_off, P.f_ncnt, P.f_wcnt, P.work);
    LENS_LAUNCHED("k_work_count");
  }
  int64_t nseam = 0;
  Scratch seam = eval32_fused(P, g, rect.as<int64_t>(), edge, ip, map32, rowdiff, stats_dev, rq,
                              rqcount, nseam, s);
  // the cells on leaves' last corner rows and columns, from the boundary corners
  ipm_accumulate_list(edge, g.nx, seam.as<int>(), nseam, ip, map32, rowdiff, stats_dev, queue,
                      qcount, rq, rqcount, s, P.timing ? &P.ev_ipm : nullptr);
}

void evaluate_grid(Plan& P, const GridRows& g, double* y, double* jac, cudaStream_t s) {
  grid_impl<false>(P, g, y, jac, nullptr, nullptr, s);
}

void evaluate_grid_pix(Plan& P, const GridRows& g, PixCorner* out, const IpmParams& ip,
                       cudaStream_t s) {
  grid_impl<true>(P, g, nullptr, nullptr, out, &ip, s);
}

void bucket_rays(Plan& P, const double* rays, int64_t m, int tile, RayBuckets& B, cudaStream_t s) {
  const int64_t nl = P.n_active_leaves;
  if (nl == 0) fail(LENS_EDOMAIN, "plan has no active leaves");
  Scratch slot(&P.da, sizeof(int) * m);
  Scratch cnt(&P.da, sizeof(int64_t) * (nl + 1));
  Scratch cur(&P.da, sizeof(int64_t) * (nl + 1));
  Scratch tiles(&P.da, sizeof(int64_t) * (nl + 1));
  Scratch err(&P.da, sizeof(int) * 4);
  B.off = Scratch(&P.da, sizeof(int64_t) * (nl + 1));
  B.perm = Scratch(&P.da, sizeof(int) * m);
  B.toff = Scratch(&P.da, sizeof(int64_t) * (nl + 1));
  LENS_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes, s));
  LENS_CUDA(cudaMemsetAsync(cur.p, 0, cur.bytes, s));
  LENS_CUDA(cudaMemsetAsync(err.p, 0, err.bytes, s));
  const double scale = (double)(1ull << P.depth) / P.root_size;
  k_ray_leaf<<<grid_for(m, 256), 256, 0, s>>>(rays, m, P.box_child, P.box_lidx, P.root_lo[0],
                                              P.root_lo[1], scale, P.depth, slot.as<int>(),
                                              cnt.as<int64_t>(), err.as<int>());
  LENS_LAUNCHED("k_ray_leaf");
  exclusive_scan_i64(cnt.as<int64_t>(), B.off.as<int64_t>(), nl + 1, P.da, s);
  k_ray_scatter<<<grid_for(m, 256), 256, 0, s>>>(slot.as<int>(), m, B.off.as<int64_t>(),
                                                 cur.as<int64_t>(), B.perm.as<int>());
  LENS_LAUNCHED("k_ray_scatter");
  k_tiles_from_counts<<<grid_for(nl + 1, 256), 256, 0, s>>>(cnt.as<int64_t>(), nl + 1, tile,
                                                            tiles.as<int64_t>());
  LENS_LAUNCHED("k_tiles_from_counts");
  exclusive_scan_i64(tiles.as<int64_t>(), B.toff.as<int64_t>(), nl + 1, P.da, s);
  int herr[4] = {0, 0, 0, 0};
  B.total = 0;
  LENS_CUDA(cudaMemcpyAsync(&B.total, B.toff.as<int64_t>() + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaMemcpyAsync(herr, err.p, sizeof(herr), cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaStreamSynchronize(s));
  if (herr[0]) fail(LENS_EDOMAIN, "a ray lies outside the plan's target region (or is not finite)");
}

void evaluate_rays(Plan& P, const double* rays, int64_t m, double* y, double* jac, cudaStream_t s) {
  if (m == 0) return;
  RayBuckets B;
  bucket_rays(P, rays, m, tile_rays(P), B, s);
  Scratch tl = tile_leaves(P, B.toff.as<int64_t>(), P.n_active_leaves, B.total, s);
  if (P.prec == LENS_FP32_BULK) {
    eval32_rays(P, rays, B.off.as<int64_t>(), B.perm.as<int>(), tl.as<int2>(), B.total, y, jac, s);
    return;
  }
  wait_expansions(P, s);
  EvalArgs A = base_args(P);
  A.tile_leaf = tl.as<int2>();
  A.rays = rays; A.ray_off = B.off.as<int64_t>(); A.perm = B.perm.as<int>();
  A.y = y; A.jac = jac;
  launch_eval<false, false>(P, A, B.total, jac != nullptr, s);
}

}  // namespace lens
