// Launch wrappers of the quartet kernels for one (bra class X, ket class Y).
// Each eri_inst_XY.cu instantiates them for FP64 and FP32 so that the 21
// class pairs compile in parallel.
#pragma once
#include <algorithm>

#include "fsim_internal.h"

namespace fsim {

// Persistent launch: grid = min(work items, resident CTAs on the device).
int device_sm_count();

template <typename Real, int X, int Y>
cudaError_t launch_jk(const JKParams<Real>& p, cudaStream_t s) {
  constexpr int LA = pair_cls_la(X), LB = pair_cls_lb(X), LC = pair_cls_la(Y), LD = pair_cls_lb(Y);
  constexpr int CS = chunk_size<Real>(X, Y);
  using BC = PairCls<LA, LB>;
  static_assert((size_t)(CS + 1) * BC::NC * kJKThreads * sizeof(Real) <= kJKBlockSmemMax,
                "per-thread quartet blocks exceed the shared-memory budget");
  auto k = jk_kernel<Real, LA, LB, LC, LD, CS>;
  const size_t smem = jk_smem_bytes<Real, LA, LB, CS>(p.bra_ppmax);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (p.nitems == 0) return cudaSuccess;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kJKThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(p.nitems, std::max(1, occ) * device_sm_count());
  k<<<grid, kJKThreads, smem, s>>>(p);
  return cudaGetLastError();
}

#define FSIM_INSTANTIATE_JK(T, X, Y) template cudaError_t launch_jk<T, X, Y>(const JKParams<T>&, cudaStream_t);

}  // namespace fsim
