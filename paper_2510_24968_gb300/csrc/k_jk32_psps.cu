// Kernel instantiation: jk32, (ps|ps) class pair.
#include "eri_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JK(float, 1, 1)
}  // namespace fsim
