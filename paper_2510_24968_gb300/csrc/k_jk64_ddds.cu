// Kernel instantiation: jk64, (dd|ds) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 5, 3)
}  // namespace fsim
