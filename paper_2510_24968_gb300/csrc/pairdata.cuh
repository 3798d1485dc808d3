// Shell-pair data kernel (paper Sec. 2.1.3 Eqs. recurrence-A/B, Sec. 2.4):
// shared by basis.cu (s/p/d classes) and k_pairdata_f.cu (f classes), which
// compile in parallel.
#pragma once
#include "fsim_internal.h"

namespace fsim {

// One thread per (pair, primitive pair): p, P and the non-zero E^{ab}_{tuv}
// with the contraction coefficients and normalisation folded in.
__host__ __device__ constexpr double odd_dfact(int i) {  // (2i-1)!! for i = 0..3
  return i == 2 ? 3.0 : (i == 3 ? 15.0 : 1.0);
}
__host__ __device__ constexpr double comp_norm(int l, int c) {
  // 1/sqrt((2i-1)!!(2j-1)!!(2k-1)!!) of component (i, j, k), l <= 3
  return 1.0 / sqrt(odd_dfact(cart_comp(l, c, 0)) * odd_dfact(cart_comp(l, c, 1)) * odd_dfact(cart_comp(l, c, 2)));
}

template <int LA, int LB>
__global__ void pair_data_kernel(int n, int ppmax, const int4* __restrict__ idx, const double* __restrict__ cen,
                                 const double* __restrict__ alpha, const double* __restrict__ coef,
                                 const int* __restrict__ nprim, double* __restrict__ pd64,
                                 float* __restrict__ pd32, double4_32a* __restrict__ pq64, float4* __restrict__ pq32) {
  using PC = PairCls<LA, LB>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ppmax) return;
  const int j = t % n, k = t / n;
  const int4 pi = idx[j];
  const int sa = pi.z, sb = pi.w;
  const int Ka = nprim[sa], Kb = nprim[sb];
  const size_t fs = (size_t)ppmax * n;
  auto put = [&](int f, double v) {
    pd64[f * fs + (size_t)k * n + j] = v;
    pd32[f * fs + (size_t)k * n + j] = (float)v;
  };
  if (k >= Ka * Kb) {
    pq64[(size_t)k * n + j] = make_double4_32a(1.0, 0.0, 0.0, 0.0);
    pq32[(size_t)k * n + j] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    put(0, 1.0);
    put(1, 0.0); put(2, 0.0); put(3, 0.0);
    for (int z = 0; z < PC::NNZ; ++z) put(4 + z, 0.0);
    return;
  }
  const int ka = k / Kb, kb = k % Kb;
  const double a = alpha[sa * kMaxPrim + ka], b = alpha[sb * kMaxPrim + kb];
  const double p = a + b, mu = a * b / p;
  double E[3][LA + 1][LB + 1][LA + LB + 1];
  double P[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const double A = cen[3 * sa + x], B = cen[3 * sb + x];
    P[x] = (a * A + b * B) / p;
    const double XAB = A - B, XPA = P[x] - A, XPB = P[x] - B, i2p = 0.5 / p;
#pragma unroll
    for (int i = 0; i <= LA; ++i)
#pragma unroll
      for (int jj = 0; jj <= LB; ++jj)
#pragma unroll
        for (int tt = 0; tt <= LA + LB; ++tt) E[x][i][jj][tt] = 0.0;
    E[x][0][0][0] = exp(-mu * XAB * XAB);
#pragma unroll
    for (int i = 1; i <= LA; ++i)
#pragma unroll
      for (int tt = 0; tt <= i; ++tt)
        E[x][i][0][tt] = (tt > 0 ? i2p * E[x][i - 1][0][tt - 1] : 0.0) + XPA * E[x][i - 1][0][tt] +
                         (tt + 1 <= i - 1 ? (tt + 1) * E[x][i - 1][0][tt + 1] : 0.0);
#pragma unroll
    for (int jj = 1; jj <= LB; ++jj)
#pragma unroll
      for (int i = 0; i <= LA; ++i)
#pragma unroll
        for (int tt = 0; tt <= i + jj; ++tt)
          E[x][i][jj][tt] = (tt > 0 ? i2p * E[x][i][jj - 1][tt - 1] : 0.0) + XPB * E[x][i][jj - 1][tt] +
                            (tt + 1 <= i + jj - 1 ? (tt + 1) * E[x][i][jj - 1][tt + 1] : 0.0);
  }
  // sqrt(2) pi^{5/4} / p folds half of 2 pi^{5/2} / (p q) into each pair
  const double scale = coef[sa * kMaxPrim + ka] * coef[sb * kMaxPrim + kb] * 1.41421356237309504880 *
                       4.18251339837959907596 /* pi^{5/4} */ / p;
  put(0, p);
  put(1, P[0]); put(2, P[1]); put(3, P[2]);
  pq64[(size_t)k * n + j] = make_double4_32a(p, P[0], P[1], P[2]);
  pq32[(size_t)k * n + j] = make_float4((float)p, (float)P[0], (float)P[1], (float)P[2]);
  static_for<PC::NC>([&](auto Aa) {
    constexpr int ac = decltype(Aa)::value;
    constexpr int ia = ac / PC::NB, ib = ac % PC::NB;
    constexpr int ix = cart_comp(LA, ia, 0), iy = cart_comp(LA, ia, 1), iz = cart_comp(LA, ia, 2);
    constexpr int jx = cart_comp(LB, ib, 0), jy = cart_comp(LB, ib, 1), jz = cart_comp(LB, ib, 2);
    const double f = scale * comp_norm(LA, ia) * comp_norm(LB, ib);
    static_for<PC::nnz(ac)>([&](auto Kk) {
      constexpr int kk = decltype(Kk)::value;
      constexpr int tt = PC::nz_t(ac, kk), uu = PC::nz_u(ac, kk), vv = PC::nz_v(ac, kk);
      put(4 + PC::off(ac) + kk, f * E[0][ix][jx][tt] * E[1][iy][jy][uu] * E[2][iz][jz][vv]);
    });
  });
}


cudaError_t launch_pair_data_f(int cls, int n, int ppmax, const int4* idx, const fsim_basis* b, double* pd64,
                               float* pd32, double4_32a* pq64, float4* pq32);

}  // namespace fsim
