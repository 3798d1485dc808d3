// Kernel instantiation: jk32, (dd|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 5, 2)
}  // namespace fsim
