// sort.cu -- LSD radix sort of 64-bit keys (+ optional 32-bit values) and
// device-wide exclusive scans.  The sort puts the stars in Morton order for
// the quadtree build (Appendix A, step 1); the scans size the build's lists.
//
// Each 8-bit pass is reduce-then-scan: (1) per-tile digit histograms plus
// the digit totals (atomics), (2) one block per digit scans its row of the
// digit-major histogram matrix and adds the keys of smaller digits, (3) a
// stable scatter in which every warp ranks its keys with __match_any_sync,
// the block combines the per-warp counts, stages its tile in shared memory
// in digit order and writes each digit's keys out as one contiguous run.
// No kernel waits on another block, so nothing can spin: there is no
// decoupled look-back and no device-side wait.
#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kIPT = 8;   // keys per thread
constexpr int kSortTile = kSortThreads * kIPT;

__global__ void __launch_bounds__(kSortThreads)
k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int nblocks,
             uint32_t* __restrict__ hist, uint32_t* __restrict__ dtot) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int k = 0; k < kIPT; ++k) {
    int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
  if (cnt[threadIdx.x]) atomicAdd(&dtot[threadIdx.x], cnt[threadIdx.x]);
}

// Scatter offsets: hist[d][b] <- (keys with a digit below d) + (keys with
// digit d in blocks before b).  One block per digit; the digit totals come
// from the histogram pass, so no block waits on another.
constexpr int kDigitScanThreads = 512;

__global__ void __launch_bounds__(kDigitScanThreads)
k_scan_digits(uint32_t* __restrict__ hist, int nblocks, const uint32_t* __restrict__ dtot) {
  __shared__ uint32_t wsum[kDigitScanThreads / 32];
  __shared__ uint32_t carry;
  const int d = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  // keys with a smaller digit
  uint32_t below = (t < d) ? dtot[t] : 0u;
  below = __reduce_add_sync(0xffffffffu, below);
  if (lane == 0) wsum[w] = below;
  __syncthreads();
  if (t == 0) {
    uint32_t b = 0;
    for (int q = 0; q < kDigitScanThreads / 32; ++q) b += wsum[q];
    carry = b;
  }
  __syncthreads();
  uint32_t* row = hist + (int64_t)d * nblocks;
  for (int c0 = 0; c0 < nblocks; c0 += kDigitScanThreads) {
    const int i = c0 + t;
    const uint32_t v = i < nblocks ? row[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    __syncthreads();  // wsum and carry of the previous chunk are consumed
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t off = carry;
    for (int q = 0; q < w; ++q) off += wsum[q];
    if (i < nblocks) row[i] = off + x - v;
    __syncthreads();
    if (t == kDigitScanThreads - 1) carry = off + x;
  }
}

__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                int shift, int nblocks, const uint32_t* __restrict__ hist) {
  __shared__ uint32_t wcnt[kSortWarps][256];
  __shared__ uint32_t wsum[kSortWarps];
  __shared__ uint32_t dstart[256];       // per digit: its start in the tile
  __shared__ int64_t dofs[256];          // per digit: global start - start in the tile
  __shared__ uint64_t skey[kSortTile];   // the tile in digit order
  __shared__ uint32_t sval[kSortTile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = threadIdx.x; q < kSortWarps * 256; q += kSortThreads) (&wcnt[0][0])[q] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * 32 * kIPT;
  uint64_t key[kIPT];
  uint32_t val[kIPT];
  uint32_t rank[kIPT];
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < kIPT; ++k) {
    const int64_t i = base + k * 32 + lane;
    const bool ok = i < n;
    key[k] = ok ? kin[i] : 0;
    val[k] = (ok && vin) ? vin[i] : 0;
    const uint32_t d = ok ? (uint32_t)((key[k] >> shift) & 0xff) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = __popc(peers & lt_mask);
    uint32_t b0 = 0;
    if (ok) b0 = wcnt[warp][d];
    __syncwarp();
    if (ok && before == 0) wcnt[warp][d] = b0 + __popc(peers);
    __syncwarp();
    rank[k] = b0 + before;
  }
  __syncthreads();
  {
    // per digit (one thread each): exclusive prefix of the per-warp counts,
    // then the digit's start in the tile (a scan over the 256 digits' totals)
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t start = incl - run;
    for (int q = 0; q < warp; ++q) start += wsum[q];
    dstart[d] = start;
    dofs[d] = (int64_t)hist[(int64_t)d * nblocks + blockIdx.x] - (int64_t)start;
  }
  __syncthreads();
  // every key's place in the tile: its digit's start, the earlier warps' keys
  // of that digit, its rank in the warp (so the scatter stays stable)
#pragma unroll
  for (int k = 0; k < kIPT; ++k) {
    const int64_t i = base + k * 32 + lane;
    if (i >= n) continue;
    const uint32_t d = (uint32_t)((key[k] >> shift) & 0xff);
    const int p = (int)(dstart[d] + wcnt[warp][d] + rank[k]);
    skey[p] = key[k];
    sval[p] = val[k];
  }
  __syncthreads();
  const int nloc = (int)min64(kSortTile, n - (int64_t)blockIdx.x * kSortTile);
  for (int t = threadIdx.x; t < nloc; t += kSortThreads) {
    const uint64_t kk = skey[t];
    const int64_t pos = dofs[(kk >> shift) & 0xff] + t;
    kout[pos] = kk;
    if (vout) vout[pos] = sval[t];
  }
}

// ---- generic int64 exclusive scan ------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t& total) {
  // warp-level inclusive scan then across warps
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  total = sh[(blockDim.x >> 5) - 1];
  const int64_t warp_base = warp ? sh[warp - 1] : 0;
  __syncthreads();
  return warp_base + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
             int64_t* __restrict__ tile_sums) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int64_t total;
  int64_t ex = block_excl_scan(s, sh, total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ tile_off) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const int64_t add = tile_off[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads)
    if (base + k < n) out[base + k] += add;
}

}  // namespace

void radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits, DeviceAlloc& da,
                    cudaStream_t s, int lo_bit) {
  if (n <= 1 || bits <= lo_bit) return;
  const int nblocks = (int)((n + kSortTile - 1) / kSortTile);
  Scratch k2(&da, sizeof(uint64_t) * (size_t)n);
  Scratch v2(&da, vals ? sizeof(uint32_t) * (size_t)n : 0);
  Scratch hist(&da, sizeof(uint32_t) * 256 * (size_t)nblocks);
  const int npass = (bits - lo_bit + 7) / 8;
  Scratch dtot(&da, sizeof(uint32_t) * 256 * (size_t)npass);
  LENS_CUDA(cudaMemsetAsync(dtot.p, 0, dtot.bytes, s));
  uint64_t* ka = keys;
  uint64_t* kb = k2.as<uint64_t>();
  uint32_t* va = vals;
  uint32_t* vb = v2.as<uint32_t>();
  int passes = 0;
  for (int shift = lo_bit; shift < bits; shift += 8, ++passes) {
    uint32_t* dt = dtot.as<uint32_t>() + 256 * passes;
    k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(ka, n, shift, nblocks, hist.as<uint32_t>(), dt);
    LENS_LAUNCHED("k_radix_hist");
    k_scan_digits<<<256, kDigitScanThreads, 0, s>>>(hist.as<uint32_t>(), nblocks, dt);
    LENS_LAUNCHED("k_scan_digits");
    k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, nblocks,
                                                     hist.as<uint32_t>());
    LENS_LAUNCHED("k_radix_scatter");
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (passes & 1) {
    LENS_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    if (vals) LENS_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  }
}

// ---- batched read-back of int64 values ------------------------------------
namespace {
struct PickArgs {
  const int64_t* src[kMaxPick];
  int n;
};
__global__ void k_pick_i64(PickArgs a, int64_t* __restrict__ out) {
  const int i = threadIdx.x;
  if (i < a.n) out[i] = *a.src[i];
}
}  // namespace

void read_i64(const int64_t* const* addrs, int n, int64_t* host, DeviceAlloc& da, cudaStream_t s) {
  if (n <= 0) return;
  if (n > kMaxPick) fail(LENS_EINVAL, "internal: too many values in one read-back");
  PickArgs a{};
  for (int i = 0; i < n; ++i) a.src[i] = addrs[i];
  a.n = n;
  Scratch out(&da, sizeof(int64_t) * (size_t)n);
  k_pick_i64<<<1, kMaxPick, 0, s>>>(a, out.as<int64_t>());
  LENS_LAUNCHED("k_pick_i64");
  LENS_CUDA(cudaMemcpyAsync(host, out.p, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaStreamSynchronize(s));
}

// out[i] = sum_{j<i} in[j]; returns nothing (caller reads out[n-1] + in[n-1]
// if it needs the total).  in and out may alias.
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, DeviceAlloc& da,
                        cudaStream_t s) {
  if (n <= 0) return;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  Scratch sums(&da, sizeof(int64_t) * (size_t)tiles);
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums.as<int64_t>());
  LENS_LAUNCHED("k_scan_tiles");
  if (tiles > 1) {
    exclusive_scan_i64(sums.as<int64_t>(), sums.as<int64_t>(), tiles, da, s);
    k_scan_add<<<(unsigned)tiles, kScanThreads, 0, s>>>(out, n, sums.as<int64_t>());
    LENS_LAUNCHED("k_scan_add");
  }
}

}  // namespace lens
