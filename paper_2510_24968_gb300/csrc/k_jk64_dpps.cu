// Kernel instantiation: jk64, (dp|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 4, 1)
}  // namespace fsim
