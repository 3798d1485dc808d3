// Kernel instantiation: double-float, (ds|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 3, 0)
}  // namespace fsim
