// Auxiliary kernels of a solver: initial state, conversions between the
// storage format and FP64 host planes, Eq. (3) macroscopic fields, the wall
// incoming mass of Eq. (12), and FP64 reductions.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kAuxThreads = 256;

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): first output of the stream
// seeded with seed XOR counter; top 53 bits as a double in [0, 1).
__device__ __forceinline__ double splitmix_u01(uint64_t seed, uint64_t k) {
    uint64_t z = (seed ^ k) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * 0x1.0p-53;
}

// Equilibrium f~* = rho g^eq(u, T) (Eq. (4)) of every velocity, or its
// deviation w (rho g - 1) when SHIFT (drho = rho - 1 given separately so that
// it carries no cancellation error).
template <int Q, class C, bool SHIFT>
__device__ __forceinline__ void equilibrium_all(C rho, C drho, C ux, C uy, C T,
                                                const KConsts<C> &k, C (&o)[Q]) {
    // A collision with omega = 1 from f = 0 leaves exactly rho g^eq.
    Collision<Q, C, SHIFT> col;
    const C u2 = ux * ux + uy * uy;
    col.set_omega(C(1));
    col.sx = k.r * ux;
    col.sy = k.r * uy;
    col.rho = rho;
    col.set_coefficients(u2, T - C(1), rho, drho / rho, k);
    o[0] = col.rest(C(0));
    PairLoop<1, Q>::run([&](auto ic) {
        constexpr int A = decltype(ic)::value;
        col.template pair<A>(C(0), C(0), o[A], o[A + 1]);
    });
}

template <int Q, int PREC>
__device__ __forceinline__ void store_cell(typename Store<PREC>::S *f, float *rplane,
                                           const KConsts<typename Store<PREC>::C> &k, int x,
                                           int j, const typename Store<PREC>::C (&o)[Q],
                                           typename Store<PREC>::C rho) {
    using S = typename Store<PREC>::S;
    using C = typename Store<PREC>::C;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        C v = o[a];
        if constexpr (Store<PREC>::dev) v -= k.w[a] * rho;
        store_pop<S>(f, k, a, j, x, from_c<S>(v));
    }
    if constexpr (Store<PREC>::dev) store_rho(rplane, k, j, x, (float)rho);
}

// f~* = rho0 (1 + amp (2U - 1)) g^eq(0, 1) = rho w_a.
template <int Q, int PREC>
__global__ void k_init_rest(typename Store<PREC>::S *f, float *rplane,
                            const __grid_constant__ KConsts<typename Store<PREC>::C> k,
                            double rho0, double amp, uint64_t seed) {
    using C = typename Store<PREC>::C;
    const long long n = (long long)k.Nx * k.Ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / k.Nx), x = (int)(c % k.Nx);
        double rho = rho0;
        if (amp != 0.0) rho = rho0 * (1.0 + amp * (2.0 * splitmix_u01(seed, (uint64_t)c) - 1.0));
        C o[Q];
        equilibrium_all<Q, C, Store<PREC>::shifted>((C)rho, (C)(rho - 1.0), C(0), C(0), C(1), k, o);
        store_cell<Q, PREC>(f, rplane, k, x, j, o, (C)rho);
    }
}

// f~* = rho g^eq(u, T) from FP64 device planes [Ny][Nx] (NULL: u = 0, T = 1).
template <int Q, int PREC>
__global__ void k_init_fields(typename Store<PREC>::S *f, float *rplane,
                              const __grid_constant__ KConsts<typename Store<PREC>::C> k,
                              const double *rho, const double *ux, const double *uy,
                              const double *T) {
    using C = typename Store<PREC>::C;
    const long long n = (long long)k.Nx * k.Ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / k.Nx), x = (int)(c % k.Nx);
        C o[Q];
        equilibrium_all<Q, C, Store<PREC>::shifted>((C)rho[c], (C)(rho[c] - 1.0),
                                                    ux ? (C)ux[c] : C(0), uy ? (C)uy[c] : C(0),
                                                    T ? (C)T[c] : C(1), k, o);
        store_cell<Q, PREC>(f, rplane, k, x, j, o, (C)rho[c]);
    }
}

// Velocity plane a of the stored state -> FP64 logical plane [Ny][Nx].
template <int Q, int PREC>
__global__ void k_plane_to_f64(const typename Store<PREC>::S *f, const float *rplane,
                               const __grid_constant__ KConsts<typename Store<PREC>::C> k,
                               int a, double *out) {
    const long long n = (long long)k.Nx * k.Ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / k.Nx), x = (int)(c % k.Nx);
        const long long r = col_index(k, j, x) + (long long)a * k.pitch;
        double v = (double)to_c(f[r]);
        if constexpr (Store<PREC>::dev) v = (double)(to_c(f[r]) + k.w[a] * rplane[rho_index(k, j, x)]);
        if constexpr (Store<PREC>::shifted) v += (double)k.w[a];
        out[c] = v;
    }
}

// FP64 logical plane -> velocity plane a of the stored state (with images).
// BF16DEV needs the density plane written first (launch_rho_plane).
template <int Q, int PREC>
__global__ void k_plane_from_f64(typename Store<PREC>::S *f, const float *rplane,
                                 const __grid_constant__ KConsts<typename Store<PREC>::C> k,
                                 int a, const double *in) {
    using S = typename Store<PREC>::S;
    using C = typename Store<PREC>::C;
    const long long n = (long long)k.Nx * k.Ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / k.Nx), x = (int)(c % k.Nx);
        C v = (C)in[c];
        if constexpr (Store<PREC>::dev) v -= k.w[a] * rplane[rho_index(k, j, x)];
        if constexpr (Store<PREC>::shifted) v = (C)(in[c] - (double)k.w[a]);
        store_pop<S>(f, k, a, j, x, from_c<S>(v));
    }
}

// Eq. (3) fields of every cell of the stored state; T is the kinetic
// temperature sum f |c - u|^2 / (2 rho).  Per-cell arithmetic in the storage's
// compute type (FP32 or FP64), outputs FP64.  Any output may be NULL.
// acc: add the fields to the outputs instead of writing them (acc == 1), or
// write them (acc == 0).
template <int Q, int PREC>
__global__ void k_macros(const typename Store<PREC>::S *f, const float *rplane,
                         const __grid_constant__ KConsts<typename Store<PREC>::C> k,
                         double *rho, double *ux, double *uy, double *T, int acc) {
    using L = Lat<Q>;
    using C = typename Store<PREC>::C;
    const long long n = (long long)k.Nx * k.Ny;
    const C r = k.r;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / k.Nx), x = (int)(c % k.Nx);
        const long long ro = col_index(k, j, x);
        const long long rr = rho_index(k, j, x);
        C fv[Q];
        C s0 = 0, sx = 0, sy = 0, se = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            C v = to_c(f[ro + (long long)a * k.pitch]);
            if constexpr (Store<PREC>::dev) v += k.w[a] * rplane[rr];
            fv[a] = v;
            s0 += v;
            sx += C(L::ex(a)) * v;
            sy += C(L::ey(a)) * v;
            se += C(L::e2(a)) * v;
        }
        // shifted storage: the sums are of deviations; sum w = 1, sum e w = 0
        const C rh = Store<PREC>::shifted ? C(1) + s0 : s0;
        const C u = r * sx / rh, v = r * sy / rh;
        if constexpr (Store<PREC>::shifted) se += k.e2w;
        // rho D T = sum f |c - u|^2 = r^2 sum e^2 f - rho u^2
        const C e = k.r2 * se - rh * (u * u + v * v);
        const double o[4] = {(double)rh, (double)u, (double)v, (double)(e / (C(2) * rh))};
        double *out[4] = {rho, ux, uy, T};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (out[i]) out[i][c] = acc ? out[i][c] + o[i] : o[i];
        (void)fv;
    }
}

// Numerator of Eq. (12) for every ghost column of both walls: m_in[w*Nx + x].
template <int Q, int PREC>
__global__ void k_wall_mass(const typename Store<PREC>::S *f, const float *rplane,
                            const __grid_constant__ KConsts<typename Store<PREC>::C> k,
                            double *m_in) {
    using L = Lat<Q>;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * k.Nx;
         t += gridDim.x * blockDim.x) {
        const int wall = t / k.Nx, xw = t % k.Nx;
        double m = 0.0;
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            const int eyb = L::ey(b);
            if (wall == 0 ? !(eyb < 0) : !(eyb > 0)) continue;
            const int xs = wrap(xw - L::ex(b), k.Nx);
            const int depth = eyb < 0 ? -eyb : eyb;
            for (int kk = 0; kk < depth; ++kk) {
                const int row = wall == 0 ? kk : k.Ny - 1 - kk;
                double v = (double)to_c(f[col_index(k, row, xs) + (long long)b * k.pitch]);
                if constexpr (Store<PREC>::dev)
                    v += (double)k.w[b] * (double)rplane[rho_index(k, row, xs)];
                if constexpr (Store<PREC>::shifted) v += (double)k.w[b];
                m += v;
            }
        }
        m_in[t] = m;
    }
}

// Block-level FP64 sum of NV values per thread (warp shuffle, then shared).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *out) {
    __shared__ double sh[32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    if (lane == 0)
        for (int i = 0; i < NV; ++i) sh[wid][i] = v[i];
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < NV; ++i) {
            double s = lane < nw ? sh[lane][i] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) out[i] = s;
        }
    }
}

// Sum of rho over all cells: per-block partials (fixed grid, fixed order).
template <int Q, int PREC>
__global__ void k_mass_partials(const typename Store<PREC>::S *f, const float *rplane,
                                const __grid_constant__ KConsts<typename Store<PREC>::C> k,
                                double *partials) {
    // rows j = blockIdx.x, + gridDim.x, ...; the block's threads stride over x
    // (no division per cell).  FP32 / BF16DEV storage: a cell's sum of stored
    // deviations is formed in FP32 (they are small, so its rounding is far
    // below FP32 resolution of the cell's mass) and added to an FP64 total;
    // FP64 storage sums in FP64.
    double acc[1] = {0.0};
    double wsum = 0.0;
    if constexpr (Store<PREC>::dev) {
#pragma unroll
        for (int a = 0; a < Q; ++a) wsum += (double)k.w[a];
    }
    for (int j = blockIdx.x; j < k.Ny; j += gridDim.x) {
        for (int x = threadIdx.x; x < k.Nx; x += blockDim.x) {
            const typename Store<PREC>::S *cell = f + col_index(k, j, x);
            if constexpr (PREC == LBM_FP64) {
                double s = 0.0;
#pragma unroll
                for (int a = 0; a < Q; ++a) s += cell[(long long)a * k.pitch];
                acc[0] += s;
            } else {
                float sd = 0.0f;
#pragma unroll
                for (int a = 0; a < Q; ++a) sd += to_c(cell[(long long)a * k.pitch]);
                double s = (double)sd;
                if constexpr (Store<PREC>::shifted) s += 1.0;    // sum of the weights
                if constexpr (Store<PREC>::dev) s += wsum * (double)rplane[rho_index(k, j, x)];
                acc[0] += s;
            }
        }
    }
    block_sum<1>(acc, partials + blockIdx.x);
}

}  // namespace lbm
