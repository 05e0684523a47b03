// The direct step kernel's variants of the LBM_BF16DEV storage format for the 17- and
// 25-velocity lattices (the 37-velocity ones: unit_bf16_step37.cu).
#include "launchers_impl.cuh"

namespace lbm {
extern template int step_q<LBM_BF16DEV, 37>(SolverImpl &, int, int, int);
template int Launch<LBM_BF16DEV>::step(SolverImpl &, int, int, int);
template int Launch<LBM_BF16DEV>::direct_variants();
}  // namespace lbm
