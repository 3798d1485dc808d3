// Kernel instantiation: double-float, (dp|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 4, 3)
}  // namespace fsim
