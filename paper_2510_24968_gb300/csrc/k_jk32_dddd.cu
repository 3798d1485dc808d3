// Kernel instantiation: jk32, (dd|dd) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 5, 5)
}  // namespace fsim
