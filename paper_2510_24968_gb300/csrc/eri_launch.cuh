// Launch wrappers of the quartet kernels for one (bra class X, ket class Y).
// Each eri_inst_XY.cu instantiates them for FP64 and FP32 so that the 21
// class pairs compile in parallel.
#pragma once
#include <algorithm>

#include "fsim_internal.h"

namespace fsim {

// Ket components per register chunk: keep (bra comps + bra Hermite terms) x CS
// inside a register budget (FP64 counts double).
// FP64 kernels keep the whole quartet in one chunk: GB300 issues FP64 FMAs at a
// small fraction of the FP32 rate, so arrays that overflow into L1-resident
// local memory do not limit them, while chunking would repeat the Hermite
// recursion per chunk.
template <typename Real>
__host__ __device__ constexpr int chunk_size(int X, int Y) {
  const int A = ncart(pair_cls_la(X)) * ncart(pair_cls_lb(X));
  const int C = ncart(pair_cls_la(Y)) * ncart(pair_cls_lb(Y));
  const int H1 = nherm(pair_cls_la(X) + pair_cls_lb(X));
  if (sizeof(Real) == 8) return C;
  const int budget = 144;
  if ((A + H1) * C <= budget) return C;
  for (int cs = C; cs >= 1; --cs)
    if (C % cs == 0 && (A + H1) * cs <= budget * 3 / 4) return cs;
  return 1;
}

// Persistent launch: grid = min(work items, resident CTAs on the device).
int device_sm_count();

template <typename Real, int X, int Y>
cudaError_t launch_jk(const JKParams<Real>& p, cudaStream_t s) {
  constexpr int LA = pair_cls_la(X), LB = pair_cls_lb(X), LC = pair_cls_la(Y), LD = pair_cls_lb(Y);
  constexpr int CS = chunk_size<Real>(X, Y);
  using BC = PairCls<LA, LB>;
  auto k = jk_kernel<Real, LA, LB, LC, LD, CS>;
  const size_t smem = (jk_boys_smem<Real>() + 15) / 16 * 16 + (1 + kJKThreads / 32) * BC::NC * sizeof(Real) +
                      (size_t)p.bra_ppmax * (4 + BC::NNZ) * sizeof(Real);
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

// Chunk-warp launch (FP32 classes with several ket chunks); nitems counts
// (bra, 32-ket tile) pairs, the launch multiplies by the chunk groups.
template <typename Real, int X, int Y>
cudaError_t launch_jk_cw(const JKParams<Real>& p, cudaStream_t s) {
  constexpr int LA = pair_cls_la(X), LB = pair_cls_lb(X), LC = pair_cls_la(Y), LD = pair_cls_lb(Y);
  constexpr int CS = chunk_size<Real>(X, Y);
  using BC = PairCls<LA, LB>;
  using KC = PairCls<LC, LD>;
  constexpr int NGRP = (KetChunks<KC, CS>::NCH + kCWWarps - 1) / kCWWarps;
  auto k = jk_kernel_cw<Real, LA, LB, LC, LD, CS>;
  const size_t smem = (jk_boys_smem<Real>() + 15) / 16 * 16 + (1 + kCWWarps) * BC::NC * sizeof(Real) +
                      (size_t)p.bra_ppmax * (4 + BC::NNZ) * sizeof(Real);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (p.nitems == 0) return cudaSuccess;
  JKParams<Real> q = p;
  q.nitems = p.nitems * NGRP;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kJKThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(q.nitems, std::max(1, occ) * device_sm_count());
  k<<<grid, kJKThreads, smem, s>>>(q);
  return cudaGetLastError();
}

#define FSIM_INSTANTIATE_CW(X, Y) template cudaError_t launch_jk_cw<float, X, Y>(const JKParams<float>&, cudaStream_t);
#define FSIM_INSTANTIATE_JK(T, X, Y) template cudaError_t launch_jk<T, X, Y>(const JKParams<T>&, cudaStream_t);

}  // namespace fsim
