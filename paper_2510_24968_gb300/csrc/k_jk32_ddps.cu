// Kernel instantiation: jk32, (dd|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 5, 1)
}  // namespace fsim
