// AA-pattern kernel instantiations and launchers for __half population storage.
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_AA_LAUNCHERS(__half)
}  // namespace lbm
