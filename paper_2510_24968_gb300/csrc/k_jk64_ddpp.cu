// Kernel instantiation: jk64, (dd|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 5, 2)
}  // namespace fsim
