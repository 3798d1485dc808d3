// Kernel instantiation: double-float, (pp|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 2, 2)
}  // namespace fsim
