// Kernel instantiation: jk32, (pp|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 2, 0)
}  // namespace fsim
