// One-pass pull kernel of a full time step (Eq. (5) with the Eq. (12) wall).
//
// One thread per fluid cell (x, j); a block covers BX consecutive columns of
// one x-tile in RS consecutive rows (one in the fastest shapes), which each
// thread walks in order.  Every population is read once, straight from global
// memory at the source cell (x - e_ax, j - e_ay): within a tile the Q
// velocities of a row are consecutive segments and the x-halos hold the
// neighbouring tiles' columns, so a warp's 32 loads of one velocity are one
// contiguous (possibly 4..12-byte shifted) run and every source of a cell lies
// at a fixed offset ((a - e_ay Q) pitch - e_ax elements) from the cell's own
// element.  With the tile pitch a compile-time constant (PC, the pitch of
// wide grids) those offsets are immediates of the load and store
// instructions; otherwise they are per-velocity byte offsets added to the
// cell's address.  Blocks holding any of the N rows next to a wall first sum
// that wall's incoming mass M_in for the BX + 6 ghost columns their fill
// populations come from (FP64, fixed order).
#pragma once

#include <type_traits>

#include "lbm_device.cuh"

namespace lbm {

// M_in(x') for x' = x0 - 3 + t, t in [0, ncols): post-collision populations
// of the N rows next to `wall` that stream into ghost column x' (Sec. III:
// incoming at layer l when e.n < -l; summed over all layers, Eq. (12)).
template <int Q, int PREC, int BX>
__device__ __forceinline__ void wall_prologue(const typename Store<PREC>::S *__restrict__ fin,
                                              const float *__restrict__ rin,
                                              const KConsts<typename Store<PREC>::C> &k,
                                              int wall, int x0, int ncols, double *s_min) {
    using L = Lat<Q>;
    for (int t = threadIdx.x; t < ncols; t += BX) {
        const int xw = wrap(x0 - 3 + t, k.Nx);
        double m = 0.0;
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            const int eyb = L::ey(b);
            const bool incoming = wall == 0 ? (eyb < 0) : (eyb > 0);
            if (!incoming) continue;
            const int xs = wrap(xw - L::ex(b), k.Nx);
            const int depth = eyb < 0 ? -eyb : eyb;
            for (int kk = 0; kk < depth; ++kk) {
                const int row = wall == 0 ? kk : k.Ny - 1 - kk;
                double v = (double)to_c(fin[col_index(k, row, xs) + (long long)b * k.pitch]);
                if constexpr (Store<PREC>::dev)
                    v += (double)k.w[b] * (double)rin[rho_index(k, row, xs)];
                if constexpr (Store<PREC>::shifted) v += (double)k.w[b];
                m += v;
            }
        }
        s_min[t] = m;
    }
}

// Pull of cell (x, j): src is the cell's own element (velocity 0) in its
// tile, rsrc its density (BF16DEV).  PC > 0: the tile pitch, a compile-time
// constant; PC = 0: the solver's pitch, offsets from the constants.
template <int Q, int PREC, bool WALL, int PC>
__device__ __forceinline__ void pull(const typename Store<PREC>::S *__restrict__ fin,
                                     const float *__restrict__ rin,
                                     const typename Store<PREC>::S *__restrict__ src,
                                     const float *__restrict__ rsrc,
                                     const KConsts<typename Store<PREC>::C> &k, int x, int j,
                                     const double *s_min, typename Store<PREC>::C (&f)[Q]) {
    using L = Lat<Q>;
    using S = typename Store<PREC>::S;
    using C = typename Store<PREC>::C;
    StaticFor<0, Q>::run([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        const int sj = j - L::ey(a);
        if (WALL && (sj < 0 || sj >= k.Ny)) {
            const int wall = sj < 0 ? 0 : 1;
            const C spec = k.accom[wall] != 1.0
                               ? specular_source<PREC>(fin, rin, k, a, L::ex(a), x, j) : C(0);
            f[a] = wall_mix<PREC>(s_min[threadIdx.x + 3 - L::ex(a)], k.wcoef[wall][a], k.w[a],
                                  k.accom[wall], spec);
        } else {
            C v;
            if constexpr (PC > 0) {
                constexpr long long off = (long long)(a - L::ey(a) * Q) * PC - L::ex(a);
                v = to_c(ld_i<S, off * (long long)sizeof(S)>(src));
                if constexpr (Store<PREC>::dev) {
                    constexpr long long roff = -(long long)L::ey(a) * PC - L::ex(a);
                    v = dev_to_f(v, k.w[a], ld_i<float, roff * 4>(rsrc));
                }
            } else {
                v = to_c(ld_b(src, k.b_src[a]));
                if constexpr (Store<PREC>::dev) v = dev_to_f(v, k.w[a], ld_b(rsrc, k.b_rho[a]));
            }
            f[a] = v;
        }
    });
}

// Store of population A of the cell whose own element is dst (velocity 0).
template <int PC, bool CS, int A, class S, class C>
__device__ __forceinline__ void store_one(S *dst, const KConsts<C> &k, S v) {
    if constexpr (PC > 0) {
        constexpr long long off = (long long)A * PC * (long long)sizeof(S);
        if constexpr (std::is_same<S, __nv_bfloat16>::value)
            st_i<off, CS>(reinterpret_cast<unsigned short *>(dst), __bfloat16_as_ushort(v));
        else
            st_i<off, CS>(dst, v);
    } else {
        if constexpr (std::is_same<S, __nv_bfloat16>::value)
            st_b<CS>(reinterpret_cast<unsigned short *>(dst), k.b_dst[A], __bfloat16_as_ushort(v));
        else
            st_b<CS>(dst, k.b_dst[A], v);
    }
}

// Collide the pulled values f of cell (x, j) — tile t, tile column xl of a
// tile of w columns — and store the result: its own slots (dst: its element
// of velocity 0; rdst: its density, BF16DEV) and, for the kPadL columns at
// either end of the tile, the halo copies.
template <int Q, int PREC, bool CS, int PC>
__device__ __forceinline__ void collide_store(const typename Store<PREC>::C (&f)[Q],
                                              typename Store<PREC>::S *__restrict__ fout,
                                              float *__restrict__ rout,
                                              typename Store<PREC>::S *__restrict__ dst,
                                              float *__restrict__ rdst,
                                              const KConsts<typename Store<PREC>::C> &k, int t,
                                              int xl, int w, int x, int j, uint32_t seed) {
    using S = typename Store<PREC>::S;
    using C = typename Store<PREC>::C;
    const uint32_t hcell = Store<PREC>::sr ? sr_cell(seed, (uint32_t)j * (uint32_t)k.Nx + (uint32_t)x) : 0u;
    Collision<Q, C, Store<PREC>::shifted> col;
    col.setup(f, k);
    C o[Q];
    o[0] = col.rest(f[0]);
    PairLoop<1, Q>::run([&](auto ic) {
        constexpr int A = decltype(ic)::value;
        col.template pair<A>(f[A], f[A + 1], o[A], o[A + 1]);
    });

    S v[Q];
    if constexpr (Store<PREC>::sr) {
        // BF16: the rest velocity alone, then each pair (a, a + 1) rounded by
        // one conversion (the same bits as store_rounded); BF16DEV first
        // takes w_a rho off, BF16SHIFT's collision output is the deviation
        const auto dv = [&](float oa, float wa) {
            if constexpr (Store<PREC>::dev) return f_to_dev(oa, wa, col.rho);
            else return oa;
        };
        const float v0 = dv(o[0], k.w[0]);
        const uint32_t d0 = bf16x2_rounded(v0, v0, sr_word(hcell, 0));   // upper: sr_bits(h, 0)
        v[0] = __ushort_as_bfloat16((unsigned short)(d0 >> 16));
        PairLoop<1, Q>::run([&](auto ic) {
            constexpr int A = decltype(ic)::value;
            const float va = dv(o[A], k.w[A]);
            const float vb = dv(o[A + 1], k.w[A + 1]);
            const uint32_t d = bf16x2_rounded(va, vb, sr_bits_pair(hcell, A));
            v[A] = __ushort_as_bfloat16((unsigned short)(d >> 16));
            v[A + 1] = __ushort_as_bfloat16((unsigned short)d);
        });
    } else {
#pragma unroll
        for (int a = 0; a < Q; ++a) v[a] = store_rounded<S>(o[a], 0u);
    }
    StaticFor<0, Q>::run([&](auto ac) {
        constexpr int A = decltype(ac)::value;
        store_one<PC, CS, A>(dst, k, v[A]);
    });
    if constexpr (Store<PREC>::dev) *rdst = (float)col.rho;
    if (xl < kPadL || xl >= w - kPadL) {
        if (w >= 2 * kPadL) {
            // one copy, at the same offset from every velocity's slot: in the
            // previous tile's right halo (xl < kPadL) or the next tile's left
            // halo (with one tile: the periodic image x + Nx or x - Nx)
            long long d, dr;
            if (xl < kPadL) {
                const int tl = t == 0 ? k.nt - 1 : t - 1;
                const int wl = tile_width(k, tl);
                d = (tl - t) * k.tile_elems + wl;
                dr = (tl - t) * k.tile_rho + wl;
            } else {
                const int tr = t == k.nt - 1 ? 0 : t + 1;
                d = (tr - t) * k.tile_elems - w;
                dr = (tr - t) * k.tile_rho - w;
            }
            StaticFor<0, Q>::run([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                store_one<PC, CS, A>(dst + d, k, v[A]);
            });
            if constexpr (Store<PREC>::dev) rdst[dr] = (float)col.rho;
        } else {
            // a grid narrower than 2 kPadL: several images per column
            const long long rowq = (long long)j * k.Q;
#pragma unroll
            for (int a = 0; a < Q; ++a)
                store_halo_copies<S>(fout + (rowq + a) * k.pitch, k.tile_elems, k, t, xl, w, v[a]);
            if constexpr (Store<PREC>::dev)
                store_halo_copies<float>(rout + (long long)j * k.pitch, k.tile_rho, k, t, xl, w,
                                         (float)col.rho);
        }
    }
}

// BX threads per block (one row segment of a tile); MINB blocks per SM
// requested from the register allocator; CS: streaming stores; RS rows per
// block, walked in order (rows [RS blockIdx.y, RS blockIdx.y + RS)); PC: the
// tile pitch as a compile-time constant (0: the solver's).  Grid: blockIdx.x
// = tile * ceil(tw / BX) + block of the tile.
template <int Q, int PREC, int BX, int MINB, bool CS, int RS, int PC>
__global__ void __launch_bounds__(BX, MINB)
k_step_direct(const typename Store<PREC>::S *__restrict__ fin,
              typename Store<PREC>::S *__restrict__ fout, const float *__restrict__ rin,
              float *__restrict__ rout,
              const __grid_constant__ KConsts<typename Store<PREC>::C> k) {
    using L = Lat<Q>;
    using C = typename Store<PREC>::C;
    __shared__ double s_min[2][BX + 6];
    const int bpt = (k.tw + BX - 1) / BX;
    const int t = blockIdx.x / bpt, xl0 = (blockIdx.x - t * bpt) * BX;
    const int w = tile_width(k, t);
    if (xl0 >= w) return;                        // past the last tile's columns
    const int xl = xl0 + threadIdx.x, x = t * k.tw + xl;
    const int j0 = blockIdx.y * RS;
    const int j1 = min(k.Ny, j0 + RS);
    const bool bot = j0 < L::N, top = j1 > k.Ny - L::N;
    const int ncols = min(BX, w - xl0) + 6;
    if (bot) wall_prologue<Q, PREC, BX>(fin, rin, k, 0, t * k.tw + xl0, ncols, s_min[0]);
    if (top) wall_prologue<Q, PREC, BX>(fin, rin, k, 1, t * k.tw + xl0, ncols, s_min[1]);
    if (bot || top) __syncthreads();
    // BF16: step count of the stochastic rounding (block 0 advances it)
    uint32_t seed = 0;
    if constexpr (Store<PREC>::sr)
        seed = step_count(fin, k, blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0);
    if (xl >= w) return;
    const long long pitch = PC > 0 ? PC : k.pitch;
    const long long cell0 = t * k.tile_elems + xl + kPadL;
    const long long rcell0 = t * k.tile_rho + xl + kPadL;
    for (int j = j0; j < j1; ++j) {
        const long long cell = cell0 + (long long)j * Q * pitch;
        const long long rcell = rcell0 + (long long)j * pitch;
        const float *rsrc = Store<PREC>::dev ? rin + rcell : nullptr;
        float *rdst = Store<PREC>::dev ? rout + rcell : nullptr;
        C f[Q];
        if (j < L::N || j >= k.Ny - L::N)
            pull<Q, PREC, true, PC>(fin, rin, fin + cell, rsrc, k, x, j, s_min[j < L::N ? 0 : 1],
                                    f);
        else
            pull<Q, PREC, false, PC>(fin, rin, fin + cell, rsrc, k, x, j, s_min[0], f);
        collide_store<Q, PREC, CS, PC>(f, fout, rout, fout + cell, rdst, k, t, xl, w, x, j, seed);
    }
}

}  // namespace lbm
