// One-pass pull kernel of a full time step (Eq. (5) with the Eq. (12) wall),
// two adjacent cells per thread, for the FP32 and BF16DEV storage formats.
//
// Thread t of a block owns columns x = x0 + 2t and x + 1 of row j (x even).
// The two cells' values travel together: population a of both is one float2,
// and the whole collision (Eq. (3) moments, Eq. (4) equilibrium, Eq. (5)
// relaxation) runs on float2 values with Blackwell's packed FP32x2
// instructions, one FFMA2 / FMUL2 / FADD2 for both cells, in the same explicit
// operations as the one-cell kernels (bit-identical results).  A source pair
// (x - e_x, x + 1 - e_x) starts on an even column when e_x is even: then it
// is one 8-byte load (FP32) or one 4-byte load of two BF16 values; otherwise
// two loads.  The post-collision pair is one 8-byte store (FP32), or one
// 4-byte store of two BF16 values converted together by the hardware's
// stochastic-rounding conversion (cvt.rs.satfinite.bf16x2.f32) with the same
// 16 random bits per value as the one-cell kernels.  Blocks holding any of the
// N rows next to a wall first sum that wall's incoming mass for their 2 BX + 6
// ghost columns (FP64, fixed order).
#pragma once

#include "k_step_direct.cuh"

namespace lbm {

template <int PREC> struct PairIO;

// FP32 storage: deviations d = f - w, the collision's own form
template <> struct PairIO<LBM_FP32> {
    // population pair at element `e` (x even: e even iff EVEN)
    template <bool EVEN>
    __device__ __forceinline__ static float2 ld(const float *__restrict__ fin,
                                                const float *__restrict__, long long e, long long,
                                                float) {
        if constexpr (EVEN) return *reinterpret_cast<const float2 *>(fin + e);
        else return make_float2(fin[e], fin[e + 1]);
    }
    __device__ __forceinline__ static void st(float *__restrict__ fout, long long e, float2 v,
                                              float, float2, uint32_t, uint32_t, int) {
        *reinterpret_cast<float2 *>(fout + e) = v;
    }
    __device__ __forceinline__ static float one(float v, float, float, uint32_t, int) { return v; }
};

// BF16DEV storage: d = f - w rho in BF16 with the FP32 density plane
template <> struct PairIO<LBM_BF16DEV> {
    // two BF16 values as the FP32 values they hold (BF16 is the top half)
    __device__ __forceinline__ static float2 unpack(uint32_t w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    template <bool EVEN>
    __device__ __forceinline__ static float2 ld(const __nv_bfloat16 *__restrict__ fin,
                                                const float *__restrict__ rin, long long e,
                                                long long r, float w) {
        float2 d, rho;
        if constexpr (EVEN) {
            d = unpack(*reinterpret_cast<const uint32_t *>(fin + e));
            rho = *reinterpret_cast<const float2 *>(rin + r);
        } else {
            const unsigned short *u = reinterpret_cast<const unsigned short *>(fin + e);
            d = make_float2(__uint_as_float((uint32_t)u[0] << 16),
                            __uint_as_float((uint32_t)u[1] << 16));
            rho = make_float2(rin[r], rin[r + 1]);
        }
        return Ar<float2>::fma(Ar<float2>::bc(w), rho, d);      // f = d + w rho, per cell
    }
    // d = f - w rho of both cells, rounded stochastically to BF16 by one
    // conversion: cell x + 1 to the upper half with bits b1, cell x to the
    // lower half with bits b0 (the random bits of each value are the top 16
    // bits of rbits' half, as the hardware conversion uses them)
    __device__ __forceinline__ static void st(__nv_bfloat16 *__restrict__ fout, long long e,
                                              float2 v, float w, float2 rho, uint32_t h0,
                                              uint32_t h1, int a) {
        const float2 dv = Ar<float2>::fma(Ar<float2>::bc(-w), rho, v);
        const uint32_t rbits = (sr_bits(h1, a) << 16) | sr_bits(h0, a);
        uint32_t out;
        asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(out) : "f"(dv.y), "f"(dv.x), "r"(rbits));
        *reinterpret_cast<uint32_t *>(fout + e) = out;
    }
    // one cell (the edge columns), rounded as the one-cell kernels round it
    __device__ __forceinline__ static __nv_bfloat16 one(float v, float w, float rho, uint32_t h,
                                                        int a) {
        return store_rounded<__nv_bfloat16>(f_to_dev(v, w, rho), sr_bits(h, a));
    }
};

// f_in of both cells (Eq. (5) pull, Eq. (12) wall in the N rows next to a wall)
template <int Q, int PREC, bool WALL>
__device__ __forceinline__ void pull_pair(const typename Store<PREC>::S *__restrict__ fin,
                                          const float *__restrict__ rin,
                                          const KConsts<float> &k, int x, int lx, int j,
                                          const double *s_min, float2 (&f)[Q]) {
    using L = Lat<Q>;
    const int cell = j * k.pitch + x + kPadL;            // even
    StaticFor<0, Q>::run([&](auto ic) {
        constexpr int a = decltype(ic)::value;
        const int sj = j - L::ey(a);
        if (WALL && (sj < 0 || sj >= k.Ny)) {
            const int wall = sj < 0 ? 0 : 1;
            float v[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float spec = k.accom[wall] != 1.0
                                       ? specular_source<PREC>(fin, rin, k, a, L::ex(a), x + c, j)
                                       : 0.0f;
                v[c] = wall_mix<PREC>(s_min[lx + c + 3 - L::ex(a)], k.wcoef[wall][a], k.w[a],
                                      k.accom[wall], spec);
            }
            f[a] = make_float2(v[0], v[1]);
        } else {
            const long long r = cell - L::ey(a) * k.pitch - L::ex(a);
            f[a] = PairIO<PREC>::template ld<(L::ex(a) & 1) == 0>(fin, rin, (long long)k.off_src[a] + cell,
                                                                 r, k.w[a]);
        }
    });
}

// BX threads per block, 2 BX columns of one row (blockIdx.y); MINB blocks per
// SM requested from the register allocator.
template <int Q, int PREC, int BX, int MINB>
__global__ void __launch_bounds__(BX, MINB)
k_step_pair(const typename Store<PREC>::S *__restrict__ fin,
            typename Store<PREC>::S *__restrict__ fout, const float *__restrict__ rin,
            float *__restrict__ rout, const __grid_constant__ KConsts<float> k) {
    using L = Lat<Q>;
    using S = typename Store<PREC>::S;
    constexpr bool kDev = Store<PREC>::dev;
    __shared__ double s_min[2][2 * BX + 6];
    const int x0 = blockIdx.x * 2 * BX;
    const int lx = 2 * threadIdx.x;
    const int x = x0 + lx;
    const int j = blockIdx.y;
    const bool bot = j < L::N, top = j >= k.Ny - L::N;
    if (bot) wall_prologue<Q, PREC, 2 * BX, BX>(fin, rin, k, 0, x0, s_min[0]);
    if (top) wall_prologue<Q, PREC, 2 * BX, BX>(fin, rin, k, 1, x0, s_min[1]);
    if (bot || top) __syncthreads();
    uint32_t seed = 0;
    if constexpr (kDev) seed = step_count(fin, k, blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0);
    if (x >= k.Nx) return;
    // cell x + 1 beyond the last column (odd Nx): computed from in-row data
    // (the padded row holds 8 columns past Nx) and not stored
    const bool two = x + 1 < k.Nx;
    float2 f[Q];
    if (bot || top) pull_pair<Q, PREC, true>(fin, rin, k, x, lx, j, s_min[bot ? 0 : 1], f);
    else pull_pair<Q, PREC, false>(fin, rin, k, x, lx, j, s_min[0], f);

    Collision<Q, float2, Store<PREC>::shifted> col;
    col.setup(f, k);
    float2 o[Q];
    o[0] = col.rest(f[0]);
    PairLoop<1, Q>::run([&](auto ic) {
        constexpr int A = decltype(ic)::value;
        col.template pair<A>(f[A], f[A + 1], o[A], o[A + 1]);
    });

    const uint32_t cell0 = (uint32_t)j * (uint32_t)k.Nx + (uint32_t)x;
    const uint32_t h0 = kDev ? sr_cell(seed, cell0) : 0u, h1 = kDev ? sr_cell(seed, cell0 + 1u) : 0u;
    const int cell = j * k.pitch + x + kPadL;
    const bool image = x < kPadL || x + 1 >= k.Nx - kPadL;
    if (two && !image) {
#pragma unroll
        for (int a = 0; a < Q; ++a)
            PairIO<PREC>::st(fout, (long long)k.off_dst[a] + cell, o[a], k.w[a], col.rho, h0, h1, a);
        if constexpr (kDev) *reinterpret_cast<float2 *>(rout + cell) = col.rho;
    } else {
        const long long roff = (long long)j * k.pitch;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            S *row = fout + (long long)a * k.plane + roff;
            store_with_images<S>(row, x, k.Nx, PairIO<PREC>::one(o[a].x, k.w[a], col.rho.x, h0, a));
            if (two)
                store_with_images<S>(row, x + 1, k.Nx, PairIO<PREC>::one(o[a].y, k.w[a], col.rho.y, h1, a));
        }
        if constexpr (kDev) {
            store_with_images<float>(rout + roff, x, k.Nx, col.rho.x);
            if (two) store_with_images<float>(rout + roff, x + 1, k.Nx, col.rho.y);
        }
    }
}

}  // namespace lbm
