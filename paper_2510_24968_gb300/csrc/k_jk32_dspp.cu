// Kernel instantiation: jk32, (ds|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 3, 2)
}  // namespace fsim
