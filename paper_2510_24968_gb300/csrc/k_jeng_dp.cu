// Kernel instantiation: Coulomb-only (J-engine) kernels with bra class dp, all ket classes.
#include "jengine_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JENG(float, 4)
FSIM_INSTANTIATE_JENG(double, 4)
}  // namespace fsim
