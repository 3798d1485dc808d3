// Kernel instantiation: jk64, (dd|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 5, 1)
}  // namespace fsim
