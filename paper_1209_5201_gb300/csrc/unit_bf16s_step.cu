// The direct step kernel's variants of the LBM_BF16SHIFT storage format for the 17- and
// 25-velocity lattices (the 37-velocity ones: unit_bf16s_step37.cu).
#include "launchers_impl.cuh"

namespace lbm {
extern template int step_q<LBM_BF16SHIFT, 37>(SolverImpl &, int, int, int);
template int Launch<LBM_BF16SHIFT>::step(SolverImpl &, int, int, int);
template int Launch<LBM_BF16SHIFT>::direct_variants();
}  // namespace lbm
