// Kernel instantiation: double-float, (ss|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 0, 0)
}  // namespace fsim
