// Kernel instantiation: jk32, (dd|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 5, 0)
}  // namespace fsim
