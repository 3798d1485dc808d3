// Launcher of the runtime-angular-momentum quartet kernel (generic.cuh), used
// for every class pair that contains an f shell, in FP32 and FP64.
#include <algorithm>

#include "fsim_internal.h"
#include "generic.cuh"

namespace fsim {

template <typename Real>
cudaError_t launch_gen(const GenParams<Real>& p, cudaStream_t s) {
  auto k = gen_kernel<Real>;
  const size_t smem = gen_smem_bytes<Real>(p.la, p.lb, p.lc, p.ld);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess || p.nitems == 0) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kGenThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(p.nitems, std::max(1, occ) * device_sm_count());
  k<<<grid, kGenThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template cudaError_t launch_gen<float>(const GenParams<float>&, cudaStream_t);
template cudaError_t launch_gen<double>(const GenParams<double>&, cudaStream_t);

}  // namespace fsim
