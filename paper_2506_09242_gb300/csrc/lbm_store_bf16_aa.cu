// AA-pattern kernel instantiations and launchers for __nv_bfloat16 population storage.
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_AA_LAUNCHERS(__nv_bfloat16)
}  // namespace lbm
