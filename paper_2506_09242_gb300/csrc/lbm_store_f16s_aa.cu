// AA-pattern kernel instantiations and launchers for FP16 storage of h * 2^12.
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_AA_LAUNCHERS(h16s)
}  // namespace lbm
