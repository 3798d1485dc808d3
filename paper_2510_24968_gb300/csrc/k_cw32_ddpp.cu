// Kernel instantiation: chunk-warp FP32, (dd|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_CW(5, 2)
}  // namespace fsim
