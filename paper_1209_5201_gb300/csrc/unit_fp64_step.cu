// The direct step kernel's variants of the LBM_FP64 storage format for the 17- and
// 25-velocity lattices (the 37-velocity ones: unit_fp64_step37.cu).
#include "launchers_impl.cuh"

namespace lbm {
extern template int step_q<LBM_FP64, 37>(SolverImpl &, int, int, int);
template int Launch<LBM_FP64>::step(SolverImpl &, int, int, int);
template int Launch<LBM_FP64>::direct_variants();
}  // namespace lbm
