// Kernel instantiation: double-float, (ds|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 3, 2)
}  // namespace fsim
