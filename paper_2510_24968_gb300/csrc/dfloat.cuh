// Double-float arithmetic for FP64-accurate integrals on the FP32 pipe.
//
// A dfloat is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2: about 48 significant bits (relative rounding ~2^-47),
// FP32's exponent range.  The operations are built from error-free
// transformations of FP32 operations:
//   * Knuth's two-sum: s = fl(a + b), e = (a - (s - v)) + (b - v), v = s - a,
//     gives a + b = s + e exactly (6 operations);
//   * Dekker's fast two-sum for |a| >= |b|: s = fl(a + b), e = b - (s - a);
//   * the exact product with a fused multiply-add: p = fl(a b),
//     e = fma(a, b, -p), a b = p + e exactly (Dekker's product, FMA form).
// Addition adds the high parts with two-sum and the low parts in FP32, then
// renormalises: its error is a few 2^-47 of |x| + |y| (not of |x + y|), the
// same order as the propagated rounding of FP64 inputs through a cancelling
// sum at this precision.  Multiply-add x y + z costs 15 FP32 operations.
// On GB300 the FP32 pipe issues 128 lanes per SM and clock and the FP64 pipe
// 2, so a chain of dfloat multiply-adds runs several times faster than the
// same chain in FP64.
//
// Every step uses the _rn intrinsics, which the compiler never contracts into
// fused multiply-adds: a contraction inside an error-free transformation
// would count a rounding error twice.
#pragma once
#include <cuda_runtime.h>

namespace fsim {

// the FP32/FP64 fma overloads stay visible next to the dfloat one below
using ::fma;

struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit dfloat(int v) : hi((float)v), lo(0.0f) {}  // exact for |v| < 2^24
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) dfloat4 {
  dfloat x, y, z, w;
};

// Nearest dfloat to a double (host or device; constant-folded for constants).
__host__ __device__ constexpr dfloat dsplit(double d) {
  return dfloat((float)d, (float)(d - (double)(float)d));
}

__device__ __forceinline__ dfloat dsplit_rn(double d) {
  const float h = __double2float_rn(d);
  return dfloat(h, __double2float_rn(__dsub_rn(d, (double)h)));
}

__device__ __forceinline__ double to_double(dfloat x) { return __dadd_rn((double)x.hi, (double)x.lo); }

// s + e with |s| >= |e| (or s == 0) renormalised
__device__ __forceinline__ dfloat fast_two_sum(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dfloat(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float v = __fsub_rn(s, x.hi);
  float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, v)), __fsub_rn(y.hi, v));
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s, e);
}

__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }

__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// x y + z
__device__ __forceinline__ dfloat fma(dfloat x, dfloat y, dfloat z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const float s = __fadd_rn(p, z.hi);
  const float v = __fsub_rn(s, p);
  float f = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(z.hi, v));
  f = __fadd_rn(f, __fadd_rn(e, z.lo));
  return fast_two_sum(s, f);
}

__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator*=(dfloat& x, dfloat y) { return x = x * y; }

// 1/sqrt(x): the FP32 estimate r (about 22 correct bits) refined by one Newton
// step r' = r + r (1 - x r^2) / 2, which squares the relative error; x r^2 is
// formed exactly enough in dfloat that 1 - x r^2 keeps its leading bits.
__device__ __forceinline__ dfloat rsqrt_dfloat(dfloat x) {
  const float r = rsqrtf(x.hi);
  const float rr = __fmul_rn(r, r);
  const dfloat r2(rr, __fmaf_rn(r, r, -rr));
  const dfloat xr2 = x * r2;
  const float e = __fsub_rn(__fsub_rn(1.0f, xr2.hi), xr2.lo);
  return fast_two_sum(r, __fmul_rn(__fmul_rn(0.5f, r), e));
}

// loads through the read-only path and warp shuffles for the working types
__device__ __forceinline__ float ldg_r(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ldg_r(const double* p) { return __ldg(p); }
__device__ __forceinline__ dfloat ldg_r(const dfloat* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return dfloat(v.x, v.y);
}
__device__ __forceinline__ float shfl_xor_r(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor_r(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfloat shfl_xor_r(dfloat v, int o) {
  return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

}  // namespace fsim
