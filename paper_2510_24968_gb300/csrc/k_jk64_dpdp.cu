// Kernel instantiation: jk64, (dp|dp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 4, 4)
}  // namespace fsim
