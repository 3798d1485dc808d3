// Kernel instantiation: jk32, (dp|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 4, 3)
}  // namespace fsim
