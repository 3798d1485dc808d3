// Kernel instantiation: jk32, (pp|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 2, 1)
}  // namespace fsim
