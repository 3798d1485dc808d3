// Kernel instantiation: chunk-warp FP32, (dd|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_CW(5, 3)
}  // namespace fsim
