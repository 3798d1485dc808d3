// Kernel instantiation: chunk-warp FP32, (dd|dd) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_CW(5, 5)
}  // namespace fsim
