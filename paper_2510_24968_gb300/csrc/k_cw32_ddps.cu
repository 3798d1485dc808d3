// Kernel instantiation: chunk-warp FP32, (dd|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_CW(5, 1)
}  // namespace fsim
