// Kernel instantiation: Coulomb-only (J-engine) kernels with bra class dd, all ket classes.
#include "jengine_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JENG(float, 5)
FSIM_INSTANTIATE_JENG(double, 5)
}  // namespace fsim
