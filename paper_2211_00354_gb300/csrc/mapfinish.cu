// mapfinish.cu -- the end of a map (Sec. 2.3: the magnification of a pixel
// is the summed area its cells put there over the pixel area): the float32
// accumulation map plus the row prefix sums of the per-row difference array
// (the whole-pixel runs of large cells), written to the caller's float64 map
// at the end of a call and kept in float-float between chunks.
#include "cx.cuh"
#include "lens_internal.h"

namespace lens {
namespace {

// map (+)= map32 + row-wise prefix sum of the difference array, one warp per
// map row: the warp walks the row 32 columns at a time (four such groups
// loaded ahead), a shuffle scan gives each column its prefix within the
// group and a running total carries it across groups, so every load and
// store is coalesced.  The sums are float-float on the float32 pipe (about
// 48 bits; float64 adds in the scan made the flushes of an 8192^2 map bound
// by the float64 pipe), and a group whose difference entries are all zero
// skips its scan.  A flush between chunks (clear) keeps the running map as
// (hi, lo) float pairs in the float64 slots of `out` and zeroes the float32
// accumulators behind the read, so the next cells start from zero; the last
// call (clear false) adds the pairs (accumulate: there was a flush) and
// writes float64.
constexpr int kFinishThreads = 256;
constexpr int kFinishAhead = 4;

__global__ void __launch_bounds__(kFinishThreads)
k_map_finish(float* __restrict__ m32, float* __restrict__ D, int npx, int npy, int64_t ldd,
             double* __restrict__ out, bool accumulate, bool clear) {
  constexpr int kWarps = kFinishThreads / 32;
  const int lane = threadIdx.x & 31;
  const int64_t step = (int64_t)gridDim.x * kWarps;
  for (int64_t row = blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5); row < npy; row += step) {
    float* d = D + row * ldd;
    float* m = m32 + row * (int64_t)npx;
    double* o = out + row * (int64_t)npx;
    float2* pr = reinterpret_cast<float2*>(o);  // the same slots as float pairs
    ff carry{0.f, 0.f};
    for (int c0 = 0; c0 < npx; c0 += 32 * kFinishAhead) {
      float dv[kFinishAhead], mv[kFinishAhead];
      float2 av[kFinishAhead];
#pragma unroll
      for (int j = 0; j < kFinishAhead; ++j) {
        const int c = c0 + 32 * j + lane;
        const bool in = c < npx;
        dv[j] = in ? d[c] : 0.f;
        mv[j] = in ? m[c] : 0.f;
        av[j] = in && accumulate ? pr[c] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < kFinishAhead; ++j) {
        const int c = c0 + 32 * j + lane;
        ff incl{dv[j], 0.f};
        if (__any_sync(0xffffffffu, dv[j] != 0.f)) {
#pragma unroll
          for (int k = 1; k < 32; k <<= 1) {
            const float h = __shfl_up_sync(0xffffffffu, incl.hi, k);
            const float l = __shfl_up_sync(0xffffffffu, incl.lo, k);
            if (lane >= k) incl = ff_add(incl, ff{h, l});
          }
        }
        const ff base = ff_add(carry, incl);
        carry = ff_add(carry, ff{__shfl_sync(0xffffffffu, incl.hi, 31),
                                 __shfl_sync(0xffffffffu, incl.lo, 31)});
        if (c < npx) {
          ff v = ff_add(base, mv[j]);
          if (accumulate) v = ff_add(v, ff{av[j].x, av[j].y});
          if (clear) {
            pr[c] = make_float2(v.hi, v.lo);
            m[c] = 0.f;
            d[c] = 0.f;
          } else {
            o[c] = (double)v.hi + (double)v.lo;
          }
        }
      }
    }
    // column npx of the difference array only ever receives run ends
    if (clear && lane == 0) d[npx] = 0.f;
  }
}

}  // namespace

void ipm_finish_map(float* map32, float* rowdiff, int npx, int npy, double* map, bool accumulate,
                    bool clear, cudaStream_t s) {
  constexpr int kWarps = kFinishThreads / 32;
  const unsigned blocks = (unsigned)std::min<int64_t>((npy + kWarps - 1) / kWarps, 152 * 8);
  k_map_finish<<<blocks, kFinishThreads, 0, s>>>(map32, rowdiff, npx, npy, (int64_t)npx + 1, map,
                                                 accumulate, clear);
  LENS_LAUNCHED("k_map_finish");
}

}  // namespace lens
