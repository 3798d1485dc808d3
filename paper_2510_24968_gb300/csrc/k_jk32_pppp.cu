// Kernel instantiation: jk32, (pp|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 2, 2)
}  // namespace fsim
