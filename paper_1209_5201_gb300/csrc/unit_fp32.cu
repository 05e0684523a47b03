// Kernels and launchers of the LBM_FP32 storage format.
#include "launchers_impl.cuh"

namespace lbm {
template struct Launch<LBM_FP32>;
}  // namespace lbm
