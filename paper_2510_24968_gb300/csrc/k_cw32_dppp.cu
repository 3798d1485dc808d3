// Kernel instantiation: chunk-warp FP32, (dp|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_CW(4, 2)
}  // namespace fsim
