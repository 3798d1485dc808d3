// Kernel instantiation: jk64, (ds|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 3, 3)
}  // namespace fsim
