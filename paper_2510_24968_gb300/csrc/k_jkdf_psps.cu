// Kernel instantiation: double-float, (ps|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 1, 1)
}  // namespace fsim
