// Kernel instantiation: jk32, (ps|ss) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 1, 0)
}  // namespace fsim
