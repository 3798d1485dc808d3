// Kernel instantiation: jk64, (dp|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 4, 0)
}  // namespace fsim
