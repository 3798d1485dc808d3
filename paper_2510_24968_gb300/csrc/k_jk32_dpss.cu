// Kernel instantiation: jk32, (dp|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 4, 0)
}  // namespace fsim
