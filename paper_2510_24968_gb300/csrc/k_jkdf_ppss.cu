// Kernel instantiation: double-float, (pp|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 2, 0)
}  // namespace fsim
