// Kernel instantiation: jk64, (pp|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 2, 2)
}  // namespace fsim
