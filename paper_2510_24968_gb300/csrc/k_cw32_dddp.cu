// Kernel instantiation: chunk-warp FP32, (dd|dp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_CW(5, 4)
}  // namespace fsim
