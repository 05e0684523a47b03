// The direct step kernel's variants of the LBM_BF16SHIFT storage format for the
// 37-velocity lattice, with their pitch-class instantiations.
#include "launchers_impl.cuh"

namespace lbm {
template int step_q<LBM_BF16SHIFT, 37>(SolverImpl &, int, int, int);
}  // namespace lbm
