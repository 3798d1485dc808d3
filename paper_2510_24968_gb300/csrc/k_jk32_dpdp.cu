// Kernel instantiation: jk32, (dp|dp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 4, 4)
}  // namespace fsim
