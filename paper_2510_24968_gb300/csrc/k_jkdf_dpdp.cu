// Kernel instantiation: double-float, (dp|dp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 4, 4)
}  // namespace fsim
