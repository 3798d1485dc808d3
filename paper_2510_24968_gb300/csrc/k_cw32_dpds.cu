// Kernel instantiation: chunk-warp FP32, (dp|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_CW(4, 3)
}  // namespace fsim
