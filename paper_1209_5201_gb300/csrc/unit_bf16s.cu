// Kernels and launchers of the LBM_BF16SHIFT storage format but the direct step kernel
// (unit_bf16s_step.cu): one translation unit each, compiled in parallel.
#include "launchers_impl.cuh"

namespace lbm {
template int Launch<LBM_BF16SHIFT>::step_staged(SolverImpl &, int, int, int);
template int Launch<LBM_BF16SHIFT>::step_cellwarp(SolverImpl &, int, int);
template int Launch<LBM_BF16SHIFT>::staged_variants();
template int Launch<LBM_BF16SHIFT>::init_rest(SolverImpl &);
template int Launch<LBM_BF16SHIFT>::init_fields(SolverImpl &, const double *, const double *,
                                      const double *, const double *);
template int Launch<LBM_BF16SHIFT>::plane_to_f64(SolverImpl &, int, double *);
template int Launch<LBM_BF16SHIFT>::plane_from_f64(SolverImpl &, int, const double *);
template int Launch<LBM_BF16SHIFT>::macros(SolverImpl &, double *, double *, double *, double *, int);
template int Launch<LBM_BF16SHIFT>::fluxes(SolverImpl &, double *, double *, double *, double *, double *);
template int Launch<LBM_BF16SHIFT>::wall_mass(SolverImpl &, double *);
template int Launch<LBM_BF16SHIFT>::mass_partials(SolverImpl &, double *, int);
}  // namespace lbm
