// Kernel instantiation: double-float, (pp|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 2, 1)
}  // namespace fsim
