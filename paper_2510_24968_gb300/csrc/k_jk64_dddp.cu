// Kernel instantiation: jk64, (dd|dp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 5, 4)
}  // namespace fsim
