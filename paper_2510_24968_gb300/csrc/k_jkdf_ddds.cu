// Kernel instantiation: double-float, (dd|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(dfloat, 5, 3)
}  // namespace fsim
