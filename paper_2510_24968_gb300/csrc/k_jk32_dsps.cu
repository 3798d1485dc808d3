// Kernel instantiation: jk32, (ds|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 3, 1)
}  // namespace fsim
