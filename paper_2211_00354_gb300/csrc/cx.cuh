// cx.cuh -- device helpers: complex arithmetic on double2/float2, compensated
// sums, Morton interleave, binomials.  Complex numbers z = x1 + i x2 are the
// image-plane positions (Appendix A: expansions in complex form).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lens {

template <typename R> struct cx_t;
template <> struct cx_t<double> { using type = double2; };
template <> struct cx_t<float> { using type = float2; };

template <typename R> __host__ __device__ __forceinline__ typename cx_t<R>::type mk(R a, R b) {
  typename cx_t<R>::type z; z.x = a; z.y = b; return z;
}
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// a*b + c
template <typename C> __host__ __device__ __forceinline__ C cfma(C a, C b, C c) {
  C z;
  z.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
  z.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
  return z;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  float2 z;
  z.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x));
  z.y = fmaf(a.x, b.y, fmaf(a.y, b.x, c.y));
  return z;
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) {
  C z; z.x = a.x * s; z.y = a.y * s; return z;
}
// 1/z
__host__ __device__ __forceinline__ double2 cinv(double2 z) {
  double d = 1.0 / (z.x * z.x + z.y * z.y);
  return make_double2(z.x * d, -z.y * d);
}
__device__ __forceinline__ float frcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float2 cinv(float2 z) {
  float d = frcp_fast(z.x * z.x + z.y * z.y);
  return make_float2(z.x * d, -z.y * d);
}

// Error-free sum of two floats (Knuth two-sum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// Compensated accumulator (hi, lo) += x
struct fcomp {
  float hi, lo;
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Two compensated accumulators side by side (one per ray of a pair) on
// Blackwell's two-lane float32 instructions.  The error of hi + x comes from
// Dekker's fast two-sum with the operands ordered by magnitude (the ordering
// runs on the integer/compare pipe, the three paired operations on the FMA
// pipe, instead of six for Knuth's two-sum): the exact error of a rounded sum
// is unique, so the result equals fcomp::add's.  a - b is formed as
// fma(b, -1, a), exactly a - b (the product is exact, the sum rounds once).
struct fcomp2 {
  float2 hi, lo;
  __device__ __forceinline__ void add(float2 x) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const bool kx = fabsf(hi.x) >= fabsf(x.x), ky = fabsf(hi.y) >= fabsf(x.y);
    const float2 a = make_float2(kx ? hi.x : x.x, ky ? hi.y : x.y);
    const float2 b = make_float2(kx ? x.x : hi.x, ky ? x.y : hi.y);
    const float2 s = __fadd2_rn(a, b);
    const float2 e = __ffma2_rn(__ffma2_rn(a, m1, s), m1, b);  // b - (s - a)
    hi = s;
    lo = __fadd2_rn(lo, e);
  }
};

// Spread the low 32 bits of x to the even bit positions of a 64-bit word.
__host__ __device__ __forceinline__ uint64_t spread2(uint64_t x) {
  x &= 0xffffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
__host__ __device__ __forceinline__ uint32_t compact2(uint64_t x) {
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
  x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
  x = (x | (x >> 16)) & 0x00000000ffffffffull;
  return (uint32_t)x;
}
// Morton code: x bits at even, y bits at odd positions.
__host__ __device__ __forceinline__ uint64_t morton(uint32_t ix, uint32_t iy) {
  return spread2(ix) | (spread2(iy) << 1);
}

}  // namespace lens

namespace lens {
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
}  // namespace lens

namespace lens {
// ---- float-float ("double-single") arithmetic on the float32 pipe --------
// A value is hi + lo with |lo| <= ulp(hi)/2 (about 48 significant bits).  On
// GB300 the float64 pipe is ~60x slower than float32, so per-ray offsets and
// the lens-equation epilogue run in this form; float64 is used once per CTA.
struct ff {
  float hi, lo;
};
__host__ __device__ __forceinline__ ff ff_of(double x) {
  ff r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ ff ff_norm(float s, float e) {  // |s| >= |e|
  ff r;
  r.hi = s + e;
  r.lo = e - (r.hi - s);
  return r;
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return ff_norm(s, e);
}
__device__ __forceinline__ ff ff_add(ff a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e += a.lo;
  return ff_norm(s, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ff_norm(p, e);
}
__device__ __forceinline__ ff ff_mul(ff a, float b) {
  const float p = a.hi * b;
  const float e = fmaf(a.hi, b, -p) + a.lo * b;
  return ff_norm(p, e);
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// The same float-float operations on two values side by side (one per ray of
// a pair), on the two-lane float32 instructions; a - b is fma(b, -1, a), and
// -round(x*y) is round(-x*y), so every lane computes exactly what the scalar
// form computes.
struct ff2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }
__device__ __forceinline__ ff2 ff2_norm(float2 s, float2 e) {  // |s| >= |e|
  ff2 r;
  r.hi = __fadd2_rn(s, e);
  r.lo = fsub2(e, fsub2(r.hi, s));
  return r;
}
// a + b (sign = +1) or a - b (sign = -1), two-sum of the high parts
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  const float2 bb = fsub2(s, a);
  e = __fadd2_rn(fsub2(a, fsub2(s, bb)), fsub2(b, bb));
}
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2& s, float2& e) {
  s = fsub2(a, b);
  const float2 bb = fsub2(s, a);
  e = fsub2(fsub2(a, fsub2(s, bb)), __fadd2_rn(b, bb));
}
__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b) {
  float2 s, e;
  two_sum2(a.hi, b.hi, s, e);
  e = __fadd2_rn(e, __fadd2_rn(a.lo, b.lo));
  return ff2_norm(s, e);
}
__device__ __forceinline__ ff2 ff2_add(ff a, ff2 b) {  // a the same in both lanes
  return ff2_add(ff2{f2(a.hi), f2(a.lo)}, b);
}
__device__ __forceinline__ ff2 ff2_sub(ff2 a, ff2 b) {
  float2 s, e;
  two_diff2(a.hi, b.hi, s, e);
  e = __fadd2_rn(e, fsub2(a.lo, b.lo));
  return ff2_norm(s, e);
}
__device__ __forceinline__ ff2 ff2_add(ff2 a, float2 b) {
  float2 s, e;
  two_sum2(a.hi, b, s, e);
  e = __fadd2_rn(e, a.lo);
  return ff2_norm(s, e);
}
__device__ __forceinline__ ff2 ff2_sub(ff2 a, float2 b) {
  float2 s, e;
  two_diff2(a.hi, b, s, e);
  e = __fadd2_rn(e, a.lo);
  return ff2_norm(s, e);
}
__device__ __forceinline__ ff2 ff2_mul(ff a, ff2 b) {  // a the same in both lanes
  const float2 ah = f2(a.hi);
  const float2 p = __fmul2_rn(ah, b.hi);
  float2 e = __ffma2_rn(ah, b.hi, __fmul2_rn(f2(-a.hi), b.hi));  // a.hi b.hi - p, exact
  e = __ffma2_rn(ah, b.lo, __ffma2_rn(f2(a.lo), b.hi, e));
  return ff2_norm(p, e);
}
}  // namespace lens
