// Kernel instantiation: jk64, (dd|dd) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 5, 5)
}  // namespace fsim
