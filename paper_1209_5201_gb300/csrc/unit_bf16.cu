// Kernels and launchers of the LBM_BF16DEV storage format but the direct step kernel
// (unit_bf16_step.cu): one translation unit each, compiled in parallel.
#include "launchers_impl.cuh"

namespace lbm {
template int Launch<LBM_BF16DEV>::step_staged(SolverImpl &, int, int, int);
template int Launch<LBM_BF16DEV>::step_cellwarp(SolverImpl &, int, int);
template int Launch<LBM_BF16DEV>::staged_variants();
template int Launch<LBM_BF16DEV>::init_rest(SolverImpl &);
template int Launch<LBM_BF16DEV>::init_fields(SolverImpl &, const double *, const double *,
                                      const double *, const double *);
template int Launch<LBM_BF16DEV>::plane_to_f64(SolverImpl &, int, double *);
template int Launch<LBM_BF16DEV>::plane_from_f64(SolverImpl &, int, const double *);
template int Launch<LBM_BF16DEV>::macros(SolverImpl &, double *, double *, double *, double *, int);
template int Launch<LBM_BF16DEV>::fluxes(SolverImpl &, double *, double *, double *, double *, double *);
template int Launch<LBM_BF16DEV>::wall_mass(SolverImpl &, double *);
template int Launch<LBM_BF16DEV>::mass_partials(SolverImpl &, double *, int);
}  // namespace lbm
