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
// in FP64 above a caller-chosen threshold `t64` (the policy of keeping Boys in
// FP64 at large T; on GB300 FP64 issues at a small fraction of the FP32 rate,
// so that policy is an option, not the default).
#pragma once
#include <cuda_runtime.h>

namespace fsim {

constexpr int kBoysMaxN = 8;           // highest order needed: (dd|dd)
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
    double Fd[L + 1];
    boys_asymptotic<L>((double)T, Fd);
#pragma unroll
    for (int n = 0; n <= L; ++n) F[n] = (float)Fd[n];
  }
}

template <typename Real>
struct Boys;
template <>
struct Boys<double> {
  static constexpr int K = kBoysK64, NROW = kBoysN64;
  template <int L>
  static __device__ __forceinline__ void eval(double T, double (&F)[L + 1], const double* tabL, int stride,
                                              float /*t64*/) {
    boys_fp64<L>(T, F, tabL, stride);
  }
};
template <>
struct Boys<float> {
  static constexpr int K = kBoysK32, NROW = kBoysN32;
  template <int L>
  static __device__ __forceinline__ void eval(float T, float (&F)[L + 1], const float* tabL, int stride,
                                              float t64) {
    boys_fp32<L>(T, F, tabL, stride, t64);
  }
};

}  // namespace fsim
