// Kernel instantiation: double-float, (dp|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 4, 2)
}  // namespace fsim
