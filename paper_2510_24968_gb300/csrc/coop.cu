// Warp-cooperative quartet kernel instantiations (FP64 and FP32).
#include "coop.cuh"
namespace fsim {
template cudaError_t launch_coop<double>(const CoopParams<double>&, int, cudaStream_t);
template cudaError_t launch_coop<float>(const CoopParams<float>&, int, cudaStream_t);
}  // namespace fsim
