// Kernel instantiation: jk32, (ss|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 0, 0)
}  // namespace fsim
