// Kernel instantiation: double-float, (ps|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 1, 0)
}  // namespace fsim
