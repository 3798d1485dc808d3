// Kernel instantiation: Coulomb-only (J-engine) kernels with bra class ds, all ket classes.
#include "jengine_launch.cuh"
namespace fsim {
FSIM_INSTANTIATE_JENG(float, 3)
FSIM_INSTANTIATE_JENG(double, 3)
}  // namespace fsim
