// Kernel instantiation: chunk-warp FP32, (pp|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_CW(2, 2)
}  // namespace fsim
