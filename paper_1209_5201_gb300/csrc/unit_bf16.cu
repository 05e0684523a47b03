// Kernels and launchers of the LBM_BF16DEV storage format.
#include "launchers_impl.cuh"

namespace lbm {
template struct Launch<LBM_BF16DEV>;
}  // namespace lbm
