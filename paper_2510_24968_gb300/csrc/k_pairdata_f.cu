// Pair-data kernels of the four f pair classes (fs, fp, fd, ff), in their own
// translation unit so that they compile beside basis.cu.
#include "pairdata.cuh"

namespace fsim {

cudaError_t launch_pair_data_f(int cls, int n, int ppmax, const int4* idx, const fsim_basis* b, double* pd64,
                               float* pd32, double4_32a* pq64, float4* pq32) {
  const int total = n * ppmax, th = 128, bl = (total + th - 1) / th;
  if (total == 0) return cudaSuccess;
  switch (cls) {
    case 6: pair_data_kernel<3, 0><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    case 7: pair_data_kernel<3, 1><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    case 8: pair_data_kernel<3, 2><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    case 9: pair_data_kernel<3, 3><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fsim
