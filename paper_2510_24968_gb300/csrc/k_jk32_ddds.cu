// Kernel instantiation: jk32, (dd|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 5, 3)
}  // namespace fsim
