// Kernel instantiation: jk32, (dp|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 4, 1)
}  // namespace fsim
