// okey.cuh -- order-preserving integer keys of float64 values: for finite
// (and infinite) doubles, okey(a) < okey(b) exactly when a < b, so minima
// and maxima (and finiteness, from the exponent bits) are taken on the
// integer pipe -- float64 comparisons run on GB300's slow float64 pipe.
#pragma once

namespace lens {

__device__ __forceinline__ unsigned long long okey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unkey(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}
__device__ __forceinline__ bool finite_bits(double v) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

}  // namespace lens
