// Kernel instantiation: jk64, (ds|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 3, 1)
}  // namespace fsim
