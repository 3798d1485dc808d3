// Kernel instantiation: double-float, (dp|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 4, 0)
}  // namespace fsim
