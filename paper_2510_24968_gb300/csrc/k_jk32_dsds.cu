// Kernel instantiation: jk32, (ds|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 3, 3)
}  // namespace fsim
