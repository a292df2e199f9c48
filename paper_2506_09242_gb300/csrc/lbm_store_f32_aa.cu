// AA-pattern kernel instantiations and launchers for float population storage.
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_AA_LAUNCHERS(float)
}  // namespace lbm
