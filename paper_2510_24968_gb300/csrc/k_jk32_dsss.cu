// Kernel instantiation: jk32, (ds|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 3, 0)
}  // namespace fsim
