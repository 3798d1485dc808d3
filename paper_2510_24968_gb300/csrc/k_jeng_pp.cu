// Kernel instantiation: Coulomb-only (J-engine) kernels with bra class pp, all ket classes.
#include "jengine_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JENG(float, 2)
FSIM_INSTANTIATE_JENG(double, 2)
}  // namespace fsim
