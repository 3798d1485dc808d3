// Kernel instantiation: jk64, (ds|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 3, 0)
}  // namespace fsim
