// The direct step kernel's variants of the LBM_FP32 storage format for the 17- and
// 25-velocity lattices (the 37-velocity ones: unit_fp32_step37.cu).
#include "launchers_impl.cuh"

namespace lbm {
extern template int step_q<LBM_FP32, 37>(SolverImpl &, int, int, int);
template int Launch<LBM_FP32>::step(SolverImpl &, int, int, int);
template int Launch<LBM_FP32>::direct_variants();
}  // namespace lbm
