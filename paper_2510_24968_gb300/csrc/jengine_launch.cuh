// Launch wrappers of the Coulomb-only (J-engine) kernels for one ordered
// (bra class X, ket class Y); k_jeng_X.cu instantiate them per bra class for
// FP32 and FP64 so that the 36 class pairs compile in parallel.
#pragma once
#include <algorithm>

#include "fsim_internal.h"
#include "jengine.cuh"

namespace fsim {

template <typename Real, int X, int Y>
cudaError_t launch_jeng(const JEngParams<Real>& p, cudaStream_t s) {
  constexpr int LA = pair_cls_la(X), LB = pair_cls_lb(X), LC = pair_cls_la(Y), LD = pair_cls_lb(Y);
  auto k = jeng_kernel<Real, LA, LB, LC, LD>;
  const size_t smem = jeng_smem_bytes<Real, LA, LB>(p.bra_ppmax);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess || p.nitems == 0) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kJKThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(p.nitems, std::max(1, occ) * device_sm_count());
  k<<<grid, kJKThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename Real, int Y>
cudaError_t launch_jeng_rho(const PairView<Real>& ket, const Real* D, int N, Real* rho, cudaStream_t s) {
  constexpr int LC = pair_cls_la(Y), LD = pair_cls_lb(Y);
  const int n = ket.n * ket.ppmax;
  if (n == 0) return cudaSuccess;
  jeng_rho_kernel<Real, LC, LD><<<(n + 127) / 128, 128, 0, s>>>(ket, D, N, rho);
  return cudaGetLastError();
}

#define FSIM_INSTANTIATE_JENG(T, X)                                                                  \
  template cudaError_t launch_jeng<T, X, 0>(const JEngParams<T>&, cudaStream_t);                     \
  template cudaError_t launch_jeng<T, X, 1>(const JEngParams<T>&, cudaStream_t);                     \
  template cudaError_t launch_jeng<T, X, 2>(const JEngParams<T>&, cudaStream_t);                     \
  template cudaError_t launch_jeng<T, X, 3>(const JEngParams<T>&, cudaStream_t);                     \
  template cudaError_t launch_jeng<T, X, 4>(const JEngParams<T>&, cudaStream_t);                     \
  template cudaError_t launch_jeng<T, X, 5>(const JEngParams<T>&, cudaStream_t);                     \
  template cudaError_t launch_jeng_rho<T, X>(const PairView<T>&, const T*, int, T*, cudaStream_t);

}  // namespace fsim
