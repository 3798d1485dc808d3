// Kernel instantiation: Coulomb-only (J-engine) kernels with bra class ps, all ket classes.
#include "jengine_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JENG(float, 1)
FSIM_INSTANTIATE_JENG(double, 1)
}  // namespace fsim
