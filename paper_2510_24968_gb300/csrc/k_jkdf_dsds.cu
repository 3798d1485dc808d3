// Kernel instantiation: double-float, (ds|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 3, 3)
}  // namespace fsim
