// Kernel instantiation: jk32, (dd|dp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 5, 4)
}  // namespace fsim
