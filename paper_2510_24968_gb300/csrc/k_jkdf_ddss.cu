// Kernel instantiation: double-float, (dd|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 5, 0)
}  // namespace fsim
