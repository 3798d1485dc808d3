// Kernel instantiation: chunk-warp FP32, (dp|dp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_CW(4, 4)
}  // namespace fsim
