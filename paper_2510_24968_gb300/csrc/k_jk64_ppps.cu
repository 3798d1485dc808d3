// Kernel instantiation: jk64, (pp|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 2, 1)
}  // namespace fsim
