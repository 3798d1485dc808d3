// Kernel instantiation: jk64, (ss|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 0, 0)
}  // namespace fsim
