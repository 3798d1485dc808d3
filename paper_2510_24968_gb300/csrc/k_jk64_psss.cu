// Kernel instantiation: jk64, (ps|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(double, 1, 0)
}  // namespace fsim
