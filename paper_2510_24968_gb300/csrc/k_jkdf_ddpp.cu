// Kernel instantiation: double-float, (dd|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 5, 2)
}  // namespace fsim
