// Kernel instantiation: double-float, (dd|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 5, 1)
}  // namespace fsim
