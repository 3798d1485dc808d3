// Boys function F_n(T) = int_0^1 exp(-T t^2) t^{2n} dt (paper Sec. 2.3.3,
// source term of the Hermite Coulomb recursion R^n_000 = (-2a)^n F_n(a R^2)).
//
// Method (Taylor table + downward recursion, the standard grid scheme):
//   * a table F_m(T_i) on T_i = i h, built once on the host (boys_table.cpp);
//   * F_L(T) by a K-term Taylor expansion about the nearest grid point,
//       F_L(T_i + d) = sum_k F_{L+k}(T_i) (-d)^k / k!     (dF_n/dT = -F_{n+1});
//   * F_{n} = (2T F_{n+1} + e^{-T}) / (2n+1) downward to F_0 (stable);
//   * for T beyond the table, F_0 = (1/2) sqrt(pi/T) (erf = 1 to double
//     precision there) and the upward recursion F_{n+1} = ((2n+1)F_n - e^{-T})/(2T),
//     which is stable for large T.
// FP64: h = 1/16, K = 8, table to T = 36 (truncation < 1e-16 relative).
// FP32: h = 1/8, K = 5, table to T = 30; above T = 30 the asymptotic branch
// runs in FP32 (F_0 = sqrt(pi/T)/2, e^{-T} kept in the upward recursion), or
// to FP64-level accuracy above a caller-chosen threshold `t64` (the policy of
// keeping Boys in FP64 at large T).  That branch runs in double-float
// arithmetic on the FP32 pipe: F_0 = (1/2) sqrt(pi) T^{-1/2} (erfc(sqrt 30) is
// below 1e-14 of erf there) and the upward recursion in double-float, e^{-T}
// from the FP32 exponential (e^{-T} <= 9.4e-14 enters F_n, n <= 8, T >= 30, at
// most at ~1e-6 of its size, so FP32's relative error leaves ~1e-13).  The same
// branch in native FP64 made the 60-atom cloud's mixed build 4x slower on
// GB300, whose FP64 pipe issues 2 operations per clock and SM against 128 FP32.
// Double-float (dfloat): the FP64 grid and K, everything in dfloat arithmetic
// (see boys_dfloat); no FP64 operation.
#pragma once
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "md_tables.cuh"

namespace fsim {

constexpr int kBoysMaxN = 12;          // highest order needed: (ff|ff)
constexpr int kBoysK64 = 8;            // Taylor terms, FP64
constexpr int kBoysK32 = 5;            // Taylor terms, FP32
constexpr int kBoysCols = kBoysMaxN + kBoysK64 + 1;  // orders stored per grid point
constexpr double kBoysH64 = 1.0 / 16.0;
constexpr double kBoysTmax64 = 36.0;
constexpr int kBoysN64 = 577;          // 36 * 16 + 1
constexpr float kBoysH32 = 1.0f / 8.0f;
constexpr float kBoysTmax32 = 30.0f;
constexpr int kBoysN32 = 241;          // 30 * 8 + 1
constexpr double kSqrtPi = 1.7724538509055160273;

// 1/(2n+1) and 1/k as compile-time constants
__host__ __device__ constexpr double inv_odd(int n) { return 1.0 / (2 * n + 1); }
__host__ __device__ constexpr double inv_int(int k) { return 1.0 / k; }

// Large-T branch in double: F_0 = sqrt(pi/T)/2, upward recursion.
template <int L>
__device__ __forceinline__ void boys_asymptotic(double T, double (&F)[L + 1]) {
  double rT = 1.0 / T;
  F[0] = 0.5 * kSqrtPi * sqrt(rT);
  if (L > 0) {
    double e = exp(-T);
    double h = 0.5 * rT;
#pragma unroll
    for (int n = 1; n <= L; ++n) F[n] = ((2 * n - 1) * F[n - 1] - e) * h;
  }
}

// `tabL` points at column L of grid row 0; consecutive grid rows are `stride`
// apart (the full table in global memory, or only the columns L..L+K-1
// staged in shared memory).
template <int L>
__device__ __forceinline__ void boys_fp64(double T, double (&F)[L + 1], const double* __restrict__ tabL, int stride) {
  if (T < kBoysTmax64) {
    int i = __double2int_rn(T * (1.0 / kBoysH64));
    double x = i * kBoysH64 - T;  // -(T - T_i)
    const double* row = tabL + i * stride;
    double acc = row[kBoysK64 - 1];
#pragma unroll
    for (int k = kBoysK64 - 1; k >= 1; --k) acc = fma(acc, x * inv_int(k), row[k - 1]);
    F[L] = acc;
    if (L > 0) {
      double e = exp(-T);
      double T2 = 2.0 * T;
#pragma unroll
      for (int n = L - 1; n >= 0; --n) F[n] = fma(T2, F[n + 1], e) * inv_odd(n);
    }
  } else {
    boys_asymptotic<L>(T, F);
  }
}

template <int L>
__device__ __forceinline__ void boys_fp32(float T, float (&F)[L + 1], const float* __restrict__ tabL, int stride,
                                          float t64) {
  if (T < kBoysTmax32) {
    int i = __float2int_rn(T * (1.0f / kBoysH32));
    float x = i * kBoysH32 - T;
    const float* row = tabL + i * stride;
    float acc = row[kBoysK32 - 1];
#pragma unroll
    for (int k = kBoysK32 - 1; k >= 1; --k) acc = fmaf(acc, x * (float)inv_int(k), row[k - 1]);
    F[L] = acc;
    if (L > 0) {
      float e = expf(-T);
      float T2 = 2.0f * T;
#pragma unroll
      for (int n = L - 1; n >= 0; --n) F[n] = fmaf(T2, F[n + 1], e) * (float)inv_odd(n);
    }
  } else if (T < t64) {
    const float rs = rsqrtf(T);
    F[0] = 0.5f * (float)kSqrtPi * rs;
    if (L > 0) {
      const float e = expf(-T);
      const float h = 0.5f * rs * rs;
#pragma unroll
      for (int n = 1; n <= L; ++n) F[n] = ((2 * n - 1) * F[n - 1] - e) * h;
    }
  } else {
    const dfloat rs = rsqrt_dfloat(dfloat(T, 0.0f));
    dfloat Fd = dsplit(0.5 * kSqrtPi) * rs;
    F[0] = Fd.hi;  // |lo| <= ulp(hi)/2: hi is the nearest float
    if constexpr (L > 0) {
      const dfloat e(expf(-T), 0.0f);
      const dfloat rT = rs * rs;
      const dfloat h(0.5f * rT.hi, 0.5f * rT.lo);
      static_for<L>([&](auto I) {
        constexpr int n = decltype(I)::value + 1;
        Fd = (dfloat(2 * n - 1) * Fd - e) * h;
        F[n] = Fd.hi;
      });
    }
  }
}

// 1/k! as a double-float constant
__host__ __device__ constexpr double inv_fact(int k) { return k <= 1 ? 1.0 : inv_fact(k - 1) / k; }

// Double-float Boys function without FP64 operations.  `row` holds, for the
// nearest grid point T_i, F_{L..L+K-1}(T_i) and in slot K the value e^{-T_i}.
//  * T < 36: Taylor sum for F_L as in FP64; e^{-T} = e^{-T_i} e^{x},
//    x = T_i - T in [-1/32, 1/32], e^{x} by its Taylor series to x^7 (the
//    next term is below 2^-55); downward recursion.
//  * T >= 36: F_0 = (1/2) sqrt(pi) T^{-1/2} (erfc(6) < 3e-17 of it), upward
//    recursion with e^{-T} from the FP32 exponential: e^{-T} <= 2.4e-16 enters
//    F_n at most at ~1e-8 of its size (n <= 8, T >= 36), so FP32's relative
//    error leaves ~1e-15.
template <int L>
__device__ __forceinline__ void boys_dfloat(dfloat T, dfloat (&F)[L + 1], const dfloat* __restrict__ tabL,
                                            int stride) {
  if (T.hi < (float)kBoysTmax64) {
    const int i = __float2int_rn(T.hi * (float)(1.0 / kBoysH64));
    const dfloat x = dfloat((float)i * (float)kBoysH64, 0.0f) - T;  // -(T - T_i); i h is exact in FP32
    const dfloat* row = tabL + i * stride;
    dfloat acc = row[kBoysK64 - 1];
    static_for<kBoysK64 - 1>([&](auto I) {
      constexpr int k = kBoysK64 - 1 - decltype(I)::value;
      acc = fma(acc, x * dsplit(inv_int(k)), row[k - 1]);
    });
    F[L] = acc;
    if constexpr (L > 0) {
      constexpr int kExpTerms = 7;
      dfloat ex = dsplit(inv_fact(kExpTerms));
      static_for<kExpTerms>([&](auto I) {
        constexpr int k = kExpTerms - 1 - decltype(I)::value;
        ex = fma(ex, x, dsplit(inv_fact(k)));
      });
      const dfloat e = row[kBoysK64] * ex;
      const dfloat T2(2.0f * T.hi, 2.0f * T.lo);
      static_for<L>([&](auto I) {
        constexpr int n = L - 1 - decltype(I)::value;
        F[n] = fma(T2, F[n + 1], e) * dsplit(inv_odd(n));
      });
    }
  } else {
    const dfloat rs = rsqrt_dfloat(T);
    F[0] = dsplit(0.5 * kSqrtPi) * rs;
    if constexpr (L > 0) {
      const dfloat e(expf(-T.hi), 0.0f);
      const dfloat rT = rs * rs;
      const dfloat h(0.5f * rT.hi, 0.5f * rT.lo);
      static_for<L>([&](auto I) {
        constexpr int n = decltype(I)::value + 1;
        F[n] = (dfloat(2 * n - 1) * F[n - 1] - e) * h;
      });
    }
  }
}

template <typename Real>
struct Boys;
template <>
struct Boys<double> {
  static constexpr int K = kBoysK64, NROW = kBoysN64, NCOL = K;
  // table column staged in slot c (of NCOL) for class order L
  static __host__ __device__ constexpr int col(int L, int c) { return L + c; }
  template <int L>
  static __device__ __forceinline__ void eval(double T, double (&F)[L + 1], const double* tabL, int stride,
                                              float /*t64*/) {
    boys_fp64<L>(T, F, tabL, stride);
  }
};
template <>
struct Boys<float> {
  static constexpr int K = kBoysK32, NROW = kBoysN32, NCOL = K;
  static __host__ __device__ constexpr int col(int L, int c) { return L + c; }
  template <int L>
  static __device__ __forceinline__ void eval(float T, float (&F)[L + 1], const float* tabL, int stride,
                                              float t64) {
    boys_fp32<L>(T, F, tabL, stride, t64);
  }
};

template <>
struct Boys<dfloat> {
  // slots 0..K-1: F_{L..L+K-1}; slot K: e^{-T_i}, kept in the table's last
  // column, which no class order of the double-float kernels (s/p/d, L <= 8)
  // reaches (L + K - 1 <= 15 < kBoysCols - 1)
  static constexpr int K = kBoysK64, NROW = kBoysN64, NCOL = K + 1;
  static __host__ __device__ constexpr int col(int L, int c) { return c < K ? L + c : kBoysCols - 1; }
  template <int L>
  static __device__ __forceinline__ void eval(dfloat T, dfloat (&F)[L + 1], const dfloat* tabL, int stride,
                                              float /*t64*/) {
    boys_dfloat<L>(T, F, tabL, stride);
  }
};

}  // namespace fsim
