// Kernel instantiation: double-float, (ds|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 3, 1)
}  // namespace fsim
