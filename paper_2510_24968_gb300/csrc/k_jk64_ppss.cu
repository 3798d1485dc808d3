// Kernel instantiation: jk64, (pp|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 2, 0)
}  // namespace fsim
