// Kernel instantiation: Coulomb-only (J-engine) kernels with bra class ss, all ket classes.
#include "jengine_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JENG(float, 0)
FSIM_INSTANTIATE_JENG(double, 0)
}  // namespace fsim
