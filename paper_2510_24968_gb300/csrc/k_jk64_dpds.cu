// Kernel instantiation: jk64, (dp|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 4, 3)
}  // namespace fsim
