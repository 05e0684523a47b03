// Per-precision kernel launchers (host side).  Each precision is compiled in
// its own translation unit (unit_fp64.cu, unit_fp32.cu, unit_bf16.cu).
#pragma once

#include "lbm_internal.h"

namespace lbm {

template <int PREC>
struct Launch {
    static int step(SolverImpl &s, int src, int dst, int variant);   // direct kernel
    static int direct_variants();
    static int step_staged(SolverImpl &s, int src, int dst, int variant);
    static int step_cellwarp(SolverImpl &s, int src, int dst);
    static int staged_variants();
    static int init_rest(SolverImpl &s);
    static int init_fields(SolverImpl &s, const double *rho, const double *ux,
                           const double *uy, const double *T);
    static int plane_to_f64(SolverImpl &s, int a, double *out);
    static int plane_from_f64(SolverImpl &s, int a, const double *in);
    // Eq. (3) fields into FP64 device planes; acc = 1 adds them instead
    static int macros(SolverImpl &s, double *rho, double *ux, double *uy, double *T,
                      int acc = 0);
    static int fluxes(SolverImpl &s, double *sxx, double *sxy, double *syy, double *qx,
                      double *qy);
    static int wall_mass(SolverImpl &s, double *m_in);
    static int mass_partials(SolverImpl &s, double *partials, int nblocks);
};

// Precision-independent kernels (k_reduce.cu).
int launch_accumulate(cudaStream_t st, double *acc, const double *in, long long n, int first);
int launch_rho_plane(cudaStream_t st, float *rplane, const double *acc, const KConsts<float> &k);
int launch_final_sum(cudaStream_t st, const double *partials, int nblocks, int nv, double *out);
int launch_residual_partials(cudaStream_t st, const double *ux, const double *T, double *uxp,
                             double *Tp, long long n, double Tref, double *partials,
                             int nblocks);

int reduction_blocks(long long n);

}  // namespace lbm
