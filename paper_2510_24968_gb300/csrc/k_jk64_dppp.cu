// Kernel instantiation: jk64, (dp|pp) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 4, 2)
}  // namespace fsim
