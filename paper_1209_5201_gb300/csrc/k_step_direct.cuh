// One-pass pull kernel of a full time step (Eq. (5) with the Eq. (12) wall).
//
// One thread per fluid cell (x, j); a block covers BX consecutive columns of
// RS consecutive rows (one in the fastest shapes), which each thread walks in
// order.  Every population is read once, straight from global memory at the
// source cell (x - e_ax, j - e_ay): SoA rows are contiguous in x, so a warp's
// 32 loads of one velocity plane are one contiguous (possibly 4..12-byte
// shifted) segment.  Periodic images in the padded row remove the modulo in x.
// Blocks holding any of the N rows next to a wall first sum that wall's
// incoming mass M_in for the BX + 6 ghost columns their fill populations come
// from (FP64, fixed order).
#pragma once

#include <type_traits>

#include "lbm_device.cuh"

namespace lbm {

// M_in(x') for x' = x0 - 3 + t, t in [0, BX + 6): post-collision populations
// of the N rows next to `wall` that stream into ghost column x' (Sec. III:
// incoming at layer l when e.n < -l; summed over all layers, Eq. (12)).
template <int Q, int PREC, int BX>
__device__ __forceinline__ void wall_prologue(const typename Store<PREC>::S *__restrict__ fin,
                                              const float *__restrict__ rin,
                                              const KConsts<typename Store<PREC>::C> &k,
                                              int wall, int x0, double *s_min) {
    using L = Lat<Q>;
    // ghost columns x0 - 3 .. x0 + active + 2 (fewer than BX when Nx is small)
    const int ncols = min(BX, k.Nx - x0) + 6;
    for (int t = threadIdx.x; t < ncols; t += BX) {
        const int xw = wrap(x0 - 3 + t, k.Nx);
        double m = 0.0;
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            const int eyb = L::ey(b);
            const bool incoming = wall == 0 ? (eyb < 0) : (eyb > 0);
            if (!incoming) continue;
            const int xs = wrap(xw - L::ex(b), k.Nx) + kPadL;
            const int depth = eyb < 0 ? -eyb : eyb;
            for (int kk = 0; kk < depth; ++kk) {
                const int row = wall == 0 ? kk : k.Ny - 1 - kk;
                const long long idx = (long long)b * k.plane + (long long)row * k.pitch + xs;
                double v = (double)to_c(fin[idx]);
                if constexpr (Store<PREC>::dev)
                    v += (double)k.w[b] * (double)rin[(long long)row * k.pitch + xs];
                if constexpr (Store<PREC>::shifted) v += (double)k.w[b];
                m += v;
            }
        }
        s_min[t] = m;
    }
}

template <int Q, int PREC, bool WALL>
__device__ __forceinline__ void pull(const typename Store<PREC>::S *__restrict__ fin,
                                     const float *__restrict__ rin,
                                     const KConsts<typename Store<PREC>::C> &k, int x, int j,
                                     const double *s_min, typename Store<PREC>::C (&f)[Q]) {
    using L = Lat<Q>;
    using C = typename Store<PREC>::C;
    // the cell's own index; velocity a reads b_src[a] bytes from it
    const int cell = j * k.pitch + x + kPadL;
    const typename Store<PREC>::S *__restrict__ src = fin + cell;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int sj = j - L::ey(a);
        if (WALL && (sj < 0 || sj >= k.Ny)) {
            const int wall = sj < 0 ? 0 : 1;
            const C spec = k.accom[wall] != 1.0
                               ? specular_source<PREC>(fin, rin, k, a, L::ex(a), x, j) : C(0);
            f[a] = wall_mix<PREC>(s_min[threadIdx.x + 3 - L::ex(a)], k.wcoef[wall][a], k.w[a],
                                  k.accom[wall], spec);
        } else {
            C v = to_c(ld_b(src, k.b_src[a]));
            if constexpr (Store<PREC>::dev) v = dev_to_f(v, k.w[a], ld_b(rin + cell, k.b_rho[a]));
            f[a] = v;
        }
    }
}

// Collide the pulled values f of cell (x, j) and store the result.
template <int Q, int PREC, bool CS>
__device__ __forceinline__ void collide_store(const typename Store<PREC>::C (&f)[Q],
                                              typename Store<PREC>::S *__restrict__ fout,
                                              float *__restrict__ rout,
                                              const KConsts<typename Store<PREC>::C> &k, int x,
                                              int j, uint32_t seed) {
    using S = typename Store<PREC>::S;
    using C = typename Store<PREC>::C;
    const uint32_t hcell = Store<PREC>::dev ? sr_cell(seed, (uint32_t)j * (uint32_t)k.Nx + (uint32_t)x) : 0u;
    Collision<Q, C, Store<PREC>::shifted> col;
    col.setup(f, k);
    C o[Q];
    o[0] = col.rest(f[0]);
    PairLoop<1, Q>::run([&](auto ic) {
        constexpr int A = decltype(ic)::value;
        col.template pair<A>(f[A], f[A + 1], o[A], o[A + 1]);
    });

    const bool image = x < kPadL || x >= k.Nx - kPadL;
    if (!image) {
        S *__restrict__ dst = fout + (j * k.pitch + x + kPadL);
        if constexpr (Store<PREC>::dev) {
            // BF16: the rest velocity alone, then each pair (a, a + 1) rounded
            // by one conversion (the same bits as store_rounded)
            const float v0 = f_to_dev(o[0], k.w[0], col.rho);
            const uint32_t d0 = bf16x2_rounded(v0, v0, sr_word(hcell, 0));   // upper: sr_bits(h, 0)
            unsigned short *d16 = reinterpret_cast<unsigned short *>(dst);
            st_b<false>(d16, k.b_dst[0], (unsigned short)(d0 >> 16));
            PairLoop<1, Q>::run([&](auto ic) {
                constexpr int A = decltype(ic)::value;
                const float va = f_to_dev(o[A], k.w[A], col.rho);
                const float vb = f_to_dev(o[A + 1], k.w[A + 1], col.rho);
                const uint32_t d = bf16x2_rounded(va, vb, sr_bits_pair(hcell, A));
                st_b<false>(d16, k.b_dst[A], (unsigned short)(d >> 16));
                st_b<false>(d16, k.b_dst[A + 1], (unsigned short)d);
            });
            rout[j * k.pitch + x + kPadL] = (float)col.rho;
        } else {
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const S sv = store_rounded<S>(o[a], sr_bits(hcell, a));
                st_b<CS>(dst, k.b_dst[a], sv);
            }
        }
    } else {
        const long long roff = (long long)j * k.pitch;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            C v = o[a];
            if constexpr (Store<PREC>::dev) v = f_to_dev(v, k.w[a], col.rho);
            store_with_images<S>(fout + (long long)a * k.plane + roff, x, k.Nx,
                                 store_rounded<S>(v, sr_bits(hcell, a)));
        }
        if constexpr (Store<PREC>::dev) store_with_images<float>(rout + roff, x, k.Nx, (float)col.rho);
    }
}

// One cell's update: pull (in the N rows next to a wall, with the wall's
// re-emission from s_min, that wall's incoming-mass sums), collide, store.
template <int Q, int PREC, bool CS>
__device__ __forceinline__ void step_cell(const typename Store<PREC>::S *__restrict__ fin,
                                          typename Store<PREC>::S *__restrict__ fout,
                                          const float *__restrict__ rin, float *__restrict__ rout,
                                          const KConsts<typename Store<PREC>::C> &k, int x, int j,
                                          const double *s_min, uint32_t seed) {
    using L = Lat<Q>;
    using C = typename Store<PREC>::C;
    C f[Q];
    if (j < L::N || j >= k.Ny - L::N) pull<Q, PREC, true>(fin, rin, k, x, j, s_min, f);
    else pull<Q, PREC, false>(fin, rin, k, x, j, s_min, f);
    collide_store<Q, PREC, CS>(f, fout, rout, k, x, j, seed);
}

// BX threads per block (one row segment); MINB blocks per SM requested from
// the register allocator; CS: streaming stores for the interior columns; RS
// rows per block, walked in order (rows [RS blockIdx.y, RS blockIdx.y + RS)).
template <int Q, int PREC, int BX, int MINB, bool CS, int RS>
__global__ void __launch_bounds__(BX, MINB)
k_step_direct(const typename Store<PREC>::S *__restrict__ fin,
              typename Store<PREC>::S *__restrict__ fout, const float *__restrict__ rin,
              float *__restrict__ rout,
              const __grid_constant__ KConsts<typename Store<PREC>::C> k) {
    using L = Lat<Q>;
    using S = typename Store<PREC>::S;
    using C = typename Store<PREC>::C;
    __shared__ double s_min[2][BX + 6];
    const int x0 = blockIdx.x * BX;
    const int x = x0 + threadIdx.x;
    const int j0 = blockIdx.y * RS;
    const int j1 = min(k.Ny, j0 + RS);
    const bool bot = j0 < L::N, top = j1 > k.Ny - L::N;
    if (bot) wall_prologue<Q, PREC, BX>(fin, rin, k, 0, x0, s_min[0]);
    if (top) wall_prologue<Q, PREC, BX>(fin, rin, k, 1, x0, s_min[1]);
    if (bot || top) __syncthreads();
    // BF16: step count of the stochastic rounding (block 0 advances it)
    uint32_t seed = 0;
    if constexpr (Store<PREC>::dev)
        seed = step_count(fin, k, blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0);
    if (x >= k.Nx) return;
    for (int j = j0; j < j1; ++j)
        step_cell<Q, PREC, CS>(fin, fout, rin, rout, k, x, j, s_min[j < L::N ? 0 : 1], seed);
}

}  // namespace lbm
