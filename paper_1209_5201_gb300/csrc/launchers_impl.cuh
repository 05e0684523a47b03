// Definitions of Launch<PREC>: lattice dispatch and launch geometry.
#pragma once

#include "k_aux.cuh"
#include "k_fluxes.cuh"
#include "k_step_cellwarp.cuh"
#include "k_step_direct.cuh"
#include "k_step_staged.cuh"
#include "launchers.h"

namespace lbm {

template <int PREC>
struct Consts;
template <> struct Consts<LBM_FP64> {
    static const KConsts<double> &get(const SolverImpl &s) { return s.kd; }
};
template <> struct Consts<LBM_FP32> {
    static const KConsts<float> &get(const SolverImpl &s) { return s.kf; }
};
template <> struct Consts<LBM_BF16DEV> {
    static const KConsts<float> &get(const SolverImpl &s) { return s.kf; }
};
template <> struct Consts<LBM_BF16SHIFT> {
    static const KConsts<float> &get(const SolverImpl &s) { return s.kf; }
};

inline int aux_blocks(long long n) {
    long long b = (n + kAuxThreads - 1) / kAuxThreads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

#define LBM_DISPATCH_Q(Q_, ...)                                 \
    switch (Q_) {                                               \
    case 17: { constexpr int QQ = 17; __VA_ARGS__; } break;     \
    case 25: { constexpr int QQ = 25; __VA_ARGS__; } break;     \
    case 37: { constexpr int QQ = 37; __VA_ARGS__; } break;     \
    default: return (int)cudaErrorInvalidValue;                 \
    }

// ---- direct kernel variants {BX, MINB, CS, RS} ----------------------------------
// RS: rows per block
struct DirectVariants {
    static constexpr int n = 8;
    static constexpr int v[n][4] = {{128, 0, 0, 1}, {128, 7, 0, 1}, {128, 6, 0, 1}, {256, 0, 0, 1},
                                    {128, 0, 1, 1}, {192, 0, 0, 1}, {128, 0, 0, 2}, {128, 5, 0, 1}};
};

template <int Q, int PREC, int BX, int MINB, bool CS, int RS>
int launch_direct(SolverImpl &s, int src, int dst) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    // blocks of BX columns never straddle two x-tiles
    dim3 grid(k.nt * ((k.tw + BX - 1) / BX), (s.p.Ny + RS - 1) / RS);
    // a pitch class: offsets as instruction immediates (compiled for the
    // 37-velocity lattice; the others take the offsets from the constants)
    if constexpr (Q == 37 && BX == 128 && RS == 1) {
        constexpr int P0 = pitch_class(PREC, 0), P1 = pitch_class(PREC, 1),
                      P2 = pitch_class(PREC, 2);
        if (k.pitch == P0) {
            k_step_direct<Q, PREC, BX, MINB, CS, RS, P0><<<grid, BX, 0, s.stream>>>(
                (const S *)s.f[src], (S *)s.f[dst], s.rho[src], s.rho[dst], k);
            return (int)cudaGetLastError();
        }
        if (k.pitch == P1) {
            k_step_direct<Q, PREC, BX, MINB, CS, RS, P1><<<grid, BX, 0, s.stream>>>(
                (const S *)s.f[src], (S *)s.f[dst], s.rho[src], s.rho[dst], k);
            return (int)cudaGetLastError();
        }
        if (k.pitch == P2) {
            k_step_direct<Q, PREC, BX, MINB, CS, RS, P2><<<grid, BX, 0, s.stream>>>(
                (const S *)s.f[src], (S *)s.f[dst], s.rho[src], s.rho[dst], k);
            return (int)cudaGetLastError();
        }
    }
    k_step_direct<Q, PREC, BX, MINB, CS, RS, 0><<<grid, BX, 0, s.stream>>>(
        (const S *)s.f[src], (S *)s.f[dst], s.rho[src], s.rho[dst], k);
    return (int)cudaGetLastError();
}

// One lattice's direct-kernel variants (the 37-velocity ones, with their
// pitch-class instantiations, compile in a translation unit of their own).
template <int PREC, int Q>
int step_q(SolverImpl &s, int src, int dst, int variant) {
    using V = DirectVariants;
#define LBM_DIRECT_CASE(I)                                                                  \
    case I:                                                                                 \
        return launch_direct<Q, PREC, V::v[I][0], V::v[I][1], (V::v[I][2] != 0), V::v[I][3]>( \
            s, src, dst);
    switch (variant) {
        LBM_DIRECT_CASE(0)
        LBM_DIRECT_CASE(1)
        LBM_DIRECT_CASE(2)
        LBM_DIRECT_CASE(3)
        LBM_DIRECT_CASE(4)
        LBM_DIRECT_CASE(5)
        LBM_DIRECT_CASE(6)
        LBM_DIRECT_CASE(7)
    default: break;
    }
#undef LBM_DIRECT_CASE
    return (int)cudaErrorInvalidValue;
}

template <int PREC>
int Launch<PREC>::step(SolverImpl &s, int src, int dst, int variant) {
    switch (s.L.Q) {
    case 17: return step_q<PREC, 17>(s, src, dst, variant);
    case 25: return step_q<PREC, 25>(s, src, dst, variant);
    case 37: return step_q<PREC, 37>(s, src, dst, variant);
    default: break;
    }
    return (int)cudaErrorInvalidValue;
}

template <int PREC>
int Launch<PREC>::direct_variants() { return DirectVariants::n; }

template <int PREC>
int Launch<PREC>::step_cellwarp(SolverImpl &s, int src, int dst) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    const long long cells = (long long)s.p.Nx * s.p.Ny;
    if (cells > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    // programmatic dependent launch: a step's grid is launched while the
    // previous one runs and waits for it on the device (griddepcontrol.wait),
    // which hides the launch latency that dominates a step of a few thousand
    // cells
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cells);
    cfg.blockDim = dim3(32);
    cfg.stream = s.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const S *fin = (const S *)s.f[src];
    S *fout = (S *)s.f[dst];
    const float *rin = s.rho[src];
    float *rout = s.rho[dst];
    LBM_DISPATCH_Q(s.L.Q, return (int)cudaLaunchKernelEx(&cfg, k_step_cellwarp<QQ, PREC>, fin, fout,
                                                          rin, rout, k));
    return (int)cudaErrorInvalidValue;
}

// ---- TMA-staged kernel variants (tile TX x TY, ring of STAGES, CPT cells per
// consumer thread); the autotuner picks one per solver ------------------------
template <int PREC> struct Variants;
template <> struct Variants<LBM_FP32> {
    static constexpr int n = 4;
    static constexpr int v[n][4] = {{128, 2, 4, 1}, {128, 4, 2, 1}, {128, 4, 2, 2}, {64, 4, 4, 1}};
};
template <> struct Variants<LBM_FP64> {
    static constexpr int n = 2;
    static constexpr int v[n][4] = {{64, 2, 4, 1}, {64, 4, 2, 1}};
};
template <> struct Variants<LBM_BF16DEV> {
    static constexpr int n = 2;
    static constexpr int v[n][4] = {{128, 2, 4, 1}, {128, 4, 3, 1}};
};
// not built for BF16SHIFT (the direct kernel is the fast path of wide grids)
template <> struct Variants<LBM_BF16SHIFT> {
    static constexpr int n = 0;
    static constexpr int v[1][4] = {{0, 0, 0, 0}};
};

template <int Q, int PREC, int TX, int TY, int ST, int CPT>
int launch_staged(SolverImpl &s, int src, int dst) {
    using Cfg = StagedCfg<Q, PREC, TX, TY, ST, CPT>;
    using S = typename Store<PREC>::S;
    auto kern = k_step_staged<Q, PREC, TX, TY, ST, CPT>;
    int dev = 0;
    cudaGetDevice(&dev);
    static bool attr_set[64] = {false};
    if (dev < 64 && !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Cfg::kSmem);
        if (e != cudaSuccess) return (int)e;
        attr_set[dev] = true;
    }
    if (s.nt != 1) return (int)cudaErrorNotSupported;    // one x-tile grids only
    if (encode_tensor_maps(s, TX, TY)) return (int)cudaErrorInvalidValue;
    const int ntiles = ((s.p.Nx + TX - 1) / TX) * ((s.p.Ny + TY - 1) / TY);
    const int grid = ntiles < s.sm_count ? ntiles : s.sm_count;
    const auto &k = Consts<PREC>::get(s);
    kern<<<grid, Cfg::kThreads, Cfg::kSmem, s.stream>>>(
        s.tm_f[src], s.tm_r[src], (const S *)s.f[src], (S *)s.f[dst], s.rho[src], s.rho[dst],
        s.derr, k);
    return (int)cudaGetLastError();
}

template <int PREC>
int Launch<PREC>::staged_variants() { return Variants<PREC>::n; }

template <int PREC>
int Launch<PREC>::step_staged(SolverImpl &s, int src, int dst, int variant) {
    using V = Variants<PREC>;
    if (variant < 0 || variant >= V::n) return (int)cudaErrorInvalidValue;
#define LBM_VARIANT_CASE(I)                                                              \
    case I:                                                                              \
        if constexpr (I < V::n) {                                                        \
            LBM_DISPATCH_Q(s.L.Q, return (launch_staged<QQ, PREC, V::v[I][0], V::v[I][1],  \
                                                        V::v[I][2], V::v[I][3]>(s, src, dst))); \
        }                                                                                \
        break;
    switch (variant) {
        LBM_VARIANT_CASE(0)
        LBM_VARIANT_CASE(1)
        LBM_VARIANT_CASE(2)
        LBM_VARIANT_CASE(3)
    default: break;
    }
#undef LBM_VARIANT_CASE
    return (int)cudaErrorInvalidValue;
}

template <int PREC>
int Launch<PREC>::init_rest(SolverImpl &s) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    const long long n = (long long)s.p.Nx * s.p.Ny;
    LBM_DISPATCH_Q(s.L.Q, (k_init_rest<QQ, PREC><<<aux_blocks(n), kAuxThreads, 0, s.stream>>>(
                               (S *)s.f[s.cur], s.rho[s.cur], k, s.p.rho0, s.p.noise_amp,
                               s.p.seed)));
    return (int)cudaGetLastError();
}

template <int PREC>
int Launch<PREC>::init_fields(SolverImpl &s, const double *rho, const double *ux,
                              const double *uy, const double *T) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    const long long n = (long long)s.p.Nx * s.p.Ny;
    LBM_DISPATCH_Q(s.L.Q, (k_init_fields<QQ, PREC><<<aux_blocks(n), kAuxThreads, 0, s.stream>>>(
                               (S *)s.f[s.cur], s.rho[s.cur], k, rho, ux, uy, T)));
    return (int)cudaGetLastError();
}

template <int PREC>
int Launch<PREC>::plane_to_f64(SolverImpl &s, int a, double *out) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    const long long n = (long long)s.p.Nx * s.p.Ny;
    LBM_DISPATCH_Q(s.L.Q, (k_plane_to_f64<QQ, PREC><<<aux_blocks(n), kAuxThreads, 0, s.stream>>>(
                               (const S *)s.f[s.cur], s.rho[s.cur], k, a, out)));
    return (int)cudaGetLastError();
}

template <int PREC>
int Launch<PREC>::plane_from_f64(SolverImpl &s, int a, const double *in) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    const long long n = (long long)s.p.Nx * s.p.Ny;
    LBM_DISPATCH_Q(s.L.Q, (k_plane_from_f64<QQ, PREC><<<aux_blocks(n), kAuxThreads, 0, s.stream>>>(
                               (S *)s.f[s.cur], s.rho[s.cur], k, a, in)));
    return (int)cudaGetLastError();
}

template <int PREC>
int Launch<PREC>::macros(SolverImpl &s, double *rho, double *ux, double *uy, double *T,
                         int acc) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    const long long n = (long long)s.p.Nx * s.p.Ny;
    LBM_DISPATCH_Q(s.L.Q, (k_macros<QQ, PREC><<<aux_blocks(n), kAuxThreads, 0, s.stream>>>(
                               (const S *)s.f[s.cur], s.rho[s.cur], k, rho, ux, uy, T, acc)));
    return (int)cudaGetLastError();
}

template <int PREC>
int Launch<PREC>::fluxes(SolverImpl &s, double *sxx, double *sxy, double *syy, double *qx,
                         double *qy) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    dim3 grid((s.p.Nx + kFluxThreads - 1) / kFluxThreads, s.p.Ny);
    LBM_DISPATCH_Q(s.L.Q, (k_fluxes<QQ, PREC><<<grid, kFluxThreads, 0, s.stream>>>(
                               (const S *)s.f[s.cur], s.rho[s.cur], k, s.kd, sxx, sxy, syy, qx,
                               qy)));
    return (int)cudaGetLastError();
}

template <int PREC>
int Launch<PREC>::wall_mass(SolverImpl &s, double *m_in) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    LBM_DISPATCH_Q(s.L.Q, (k_wall_mass<QQ, PREC><<<aux_blocks(2LL * s.p.Nx), kAuxThreads, 0,
                                                   s.stream>>>((const S *)s.f[s.cur],
                                                               s.rho[s.cur], k, m_in)));
    return (int)cudaGetLastError();
}

template <int PREC>
int Launch<PREC>::mass_partials(SolverImpl &s, double *partials, int nblocks) {
    using S = typename Store<PREC>::S;
    const auto &k = Consts<PREC>::get(s);
    LBM_DISPATCH_Q(s.L.Q, (k_mass_partials<QQ, PREC><<<nblocks, kAuxThreads, 0, s.stream>>>(
                               (const S *)s.f[s.cur], s.rho[s.cur], k, partials)));
    return (int)cudaGetLastError();
}

}  // namespace lbm
