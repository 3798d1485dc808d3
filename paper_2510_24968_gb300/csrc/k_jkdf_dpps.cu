// Kernel instantiation: double-float, (dp|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 4, 1)
}  // namespace fsim
