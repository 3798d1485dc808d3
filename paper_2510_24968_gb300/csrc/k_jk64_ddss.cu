// Kernel instantiation: jk64, (dd|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 5, 0)
}  // namespace fsim
