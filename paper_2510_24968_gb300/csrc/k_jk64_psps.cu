// Kernel instantiation: jk64, (ps|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 1, 1)
}  // namespace fsim
