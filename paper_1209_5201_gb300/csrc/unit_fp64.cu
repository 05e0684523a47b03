// Kernels and launchers of the LBM_FP64 storage format.
#include "launchers_impl.cuh"

namespace lbm {
template struct Launch<LBM_FP64>;
}  // namespace lbm
