// Kernel instantiation: jk64, (ds|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 3, 2)
}  // namespace fsim
