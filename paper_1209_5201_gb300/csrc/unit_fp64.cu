// Kernels and launchers of the LBM_FP64 storage format but the direct step kernel
// (unit_fp64_step.cu): one translation unit each, compiled in parallel.
#include "launchers_impl.cuh"

namespace lbm {
template int Launch<LBM_FP64>::step_staged(SolverImpl &, int, int, int);
template int Launch<LBM_FP64>::step_cellwarp(SolverImpl &, int, int);
template int Launch<LBM_FP64>::staged_variants();
template int Launch<LBM_FP64>::init_rest(SolverImpl &);
template int Launch<LBM_FP64>::init_fields(SolverImpl &, const double *, const double *,
                                      const double *, const double *);
template int Launch<LBM_FP64>::plane_to_f64(SolverImpl &, int, double *);
template int Launch<LBM_FP64>::plane_from_f64(SolverImpl &, int, const double *);
template int Launch<LBM_FP64>::macros(SolverImpl &, double *, double *, double *, double *, int);
template int Launch<LBM_FP64>::fluxes(SolverImpl &, double *, double *, double *, double *, double *);
template int Launch<LBM_FP64>::wall_mass(SolverImpl &, double *);
template int Launch<LBM_FP64>::mass_partials(SolverImpl &, double *, int);
}  // namespace lbm
