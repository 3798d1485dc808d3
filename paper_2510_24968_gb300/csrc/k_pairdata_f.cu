// Pair-data kernel of the four f pair classes (fs, fp, fd, ff): the same
// quantities as pair_data_kernel (paper Sec. 2.1.3 Eqs. recurrence-A/B,
// Sec. 2.4), with the angular momenta and the non-zero enumeration as runtime
// loops.  It runs once per basis, and the unrolled form of (ff), 100
// components and 1,600 non-zeros, took longer to compile than any ERI kernel.
#include "pairdata.cuh"

namespace fsim {

namespace {

__global__ void pair_data_f_kernel(int LA, int LB, int n, int ppmax, const int4* __restrict__ idx,
                                   const double* __restrict__ cen, const double* __restrict__ alpha,
                                   const double* __restrict__ coef, const int* __restrict__ nprim,
                                   double* __restrict__ pd64, float* __restrict__ pd32,
                                   double4_32a* __restrict__ pq64, float4* __restrict__ pq32) {
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
  const int NA = ncart(LA), NB = ncart(LB);
  if (k >= Ka * Kb) {
    pq64[(size_t)k * n + j] = make_double4_32a(1.0, 0.0, 0.0, 0.0);
    pq32[(size_t)k * n + j] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    put(0, 1.0);
    put(1, 0.0); put(2, 0.0); put(3, 0.0);
    const int nnz = pair_cls_nnz(pair_cls_index(LA, LB));
    for (int z = 0; z < nnz; ++z) put(4 + z, 0.0);
    return;
  }
  const int ka = k / Kb, kb = k % Kb;
  const double a = alpha[sa * kMaxPrim + ka], b = alpha[sb * kMaxPrim + kb];
  const double p = a + b, mu = a * b / p;
  double E[3][4][4][7];  // E[axis][i][j][t], i <= LA, j <= LB, t <= i + j
  double P[3];
  for (int x = 0; x < 3; ++x) {
    const double A = cen[3 * sa + x], B = cen[3 * sb + x];
    P[x] = (a * A + b * B) / p;
    const double XAB = A - B, XPA = P[x] - A, XPB = P[x] - B, i2p = 0.5 / p;
    for (int i = 0; i <= LA; ++i)
      for (int jj = 0; jj <= LB; ++jj)
        for (int tt = 0; tt <= LA + LB; ++tt) E[x][i][jj][tt] = 0.0;
    E[x][0][0][0] = exp(-mu * XAB * XAB);
    for (int i = 1; i <= LA; ++i)
      for (int tt = 0; tt <= i; ++tt)
        E[x][i][0][tt] = (tt > 0 ? i2p * E[x][i - 1][0][tt - 1] : 0.0) + XPA * E[x][i - 1][0][tt] +
                         (tt + 1 <= i - 1 ? (tt + 1) * E[x][i - 1][0][tt + 1] : 0.0);
    for (int jj = 1; jj <= LB; ++jj)
      for (int i = 0; i <= LA; ++i)
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
  // non-zeros component after component, t-major (the order of PairCls)
  int z = 0;
  for (int ia = 0; ia < NA; ++ia)
    for (int ib = 0; ib < NB; ++ib) {
      const int ix = cart_comp(LA, ia, 0), iy = cart_comp(LA, ia, 1), iz = cart_comp(LA, ia, 2);
      const int jx = cart_comp(LB, ib, 0), jy = cart_comp(LB, ib, 1), jz = cart_comp(LB, ib, 2);
      const double f = scale * comp_norm(LA, ia) * comp_norm(LB, ib);
      for (int tt = 0; tt <= ix + jx; ++tt)
        for (int uu = 0; uu <= iy + jy; ++uu)
          for (int vv = 0; vv <= iz + jz; ++vv)
            put(4 + z++, f * E[0][ix][jx][tt] * E[1][iy][jy][uu] * E[2][iz][jz][vv]);
    }
}

}  // namespace

cudaError_t launch_pair_data_f(int cls, int n, int ppmax, const int4* idx, const fsim_basis* b, double* pd64,
                               float* pd32, double4_32a* pq64, float4* pq32) {
  const int total = n * ppmax, th = 128, bl = (total + th - 1) / th;
  if (cls < 6 || cls >= kNumPairClsAll) return cudaErrorInvalidValue;
  if (total == 0) return cudaSuccess;
  pair_data_f_kernel<<<bl, th>>>(pair_cls_la(cls), pair_cls_lb(cls), n, ppmax, idx, b->d_cen, b->d_alpha,
                                 b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32);
  return cudaGetLastError();
}

}  // namespace fsim
