// AA-pattern kernel instantiations and launchers for double population storage.
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_AA_LAUNCHERS(double)
}  // namespace lbm
