// Kernel instantiation: jk32, (dp|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 4, 2)
}  // namespace fsim
