// One-warp-per-cell form of the time step (Eq. (5) with the Eq. (12) wall),
// for grids of a few thousand cells, where the one-thread-per-cell kernel is
// bound by the latency of one thread's dependent chain (in FP64 on GB300 each
// warp instruction of that chain costs the FP64 unit's full issue time).
//
// Lane l carries velocities l and l + 32 (Q <= 37): it pulls them, the warp
// sums the moments with a butterfly of shuffles (every lane gets the totals),
// every lane forms the shell-independent Eq. (4) factors (FP64: lane s the
// coefficients of shell s, shuffled to the lanes that need them) and relaxes
// its own velocities.  Steps are launched with programmatic dependent launch.
// A wall row's warp first sums the incoming mass of the ghost columns its
// fills come from, one term per lane (the wall's term list, <= 26 terms).
// The moments are summed in another order than the one-thread kernels use,
// so results agree with them to round-off, not bit for bit.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

template <class C>
__device__ __forceinline__ C warp_allsum(C v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int Q, int PREC>
__global__ void __launch_bounds__(32)
k_step_cellwarp(const typename Store<PREC>::S *__restrict__ fin,
                typename Store<PREC>::S *__restrict__ fout, const float *__restrict__ rin,
                float *__restrict__ rout,
                const __grid_constant__ KConsts<typename Store<PREC>::C> k) {
    using L = Lat<Q>;
    using S = typename Store<PREC>::S;
    using C = typename Store<PREC>::C;
    constexpr bool SHIFT = Store<PREC>::shifted;
    // the lattice tables in shared memory, written with compile-time indices
    __shared__ int s_ex[Q], s_ey[Q], s_sh[Q];
    __shared__ int s_tb[2][32], s_tk[2][32];
    __shared__ int s_nt;
    __shared__ double s_min[7];
    const int lane = threadIdx.x;
    if (lane == 0) {
        int nb = 0, nt = 0;
        StaticFor<0, Q>::run([&](auto ic) {
            constexpr int a = decltype(ic)::value;
            s_ex[a] = L::ex(a);
            s_ey[a] = L::ey(a);
            s_sh[a] = L::sh(a);
            // incoming terms of each wall: velocity a at distance kk < |e_y|
            for (int kk = 0; kk < -L::ey(a); ++kk) { s_tb[0][nb] = a; s_tk[0][nb] = kk; ++nb; }
            for (int kk = 0; kk < L::ey(a); ++kk) { s_tb[1][nt] = a; s_tk[1][nt] = kk; ++nt; }
        });
        s_nt = nb;
    }
    __syncwarp();
    // launched with programmatic stream serialization: the previous step may
    // still be running; let the next step's launch begin, then wait for the
    // previous grid to complete (its stores visible) before touching the state
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    const int j = blockIdx.x / k.Nx, x = blockIdx.x - j * k.Nx;
    // BF16: step count of the stochastic rounding (block 0 advances it)
    uint32_t seed = 0;
    if constexpr (Store<PREC>::sr) seed = step_count(fin, k, blockIdx.x == 0 && lane == 0);
    const uint32_t hcell = Store<PREC>::sr ? sr_cell(seed, (uint32_t)blockIdx.x) : 0u;
    const bool bot = j < L::N, top = j >= k.Ny - L::N;

    // value of population a at column xc (0 <= xc < Nx) of row `row`, in the
    // collision's form
    auto load = [&](int a, int row, int xc) -> C {
        C v = to_c(fin[col_index(k, row, xc) + (long long)a * k.pitch]);
        if constexpr (Store<PREC>::dev) v = dev_to_f(v, k.w[a], rin[rho_index(k, row, xc)]);
        return v;
    };

    if (bot || top) {
        // numerator of Eq. (12) for ghost columns x - 3 .. x + 3 (FP64, one
        // term per lane, fixed butterfly order); with Nx < 7 the columns repeat
        const int wall = bot ? 0 : 1;
        const int ncol = min(7, k.Nx);
        for (int t = 0; t < 7; ++t) {
            const int xw = wrap(x - 3 + t, k.Nx);
            double m = 0.0;
            if (t < ncol) {
                if (lane < s_nt) {
                    const int b = s_tb[wall][lane], kk = s_tk[wall][lane];
                    const int row = wall == 0 ? kk : k.Ny - 1 - kk;
                    double v = (double)load(b, row, wrap(xw - s_ex[b], k.Nx));
                    if constexpr (SHIFT) v += (double)k.w[b];
                    m = v;
                }
                m = warp_allsum(m);
                if (lane == 0) s_min[t] = m;
            } else if (lane == 0) {
                s_min[t] = s_min[t % ncol];          // the same ghost column (mod Nx)
            }
            __syncwarp();
        }
    }

    auto pull = [&](int a) -> C {
        const int ex = s_ex[a], sj = j - s_ey[a];
        if (sj < 0 || sj >= k.Ny) {
            const int wall = sj < 0 ? 0 : 1;
            const C spec = k.accom[wall] != 1.0 ? specular_source<PREC>(fin, rin, k, a, ex, x, j) : C(0);
            return wall_mix<PREC>(s_min[3 - ex], k.wcoef[wall][a], k.w[a], k.accom[wall], spec);
        }
        return load(a, sj, wrap(x - ex, k.Nx));
    };
    const int a0 = lane, a1 = lane + 32;
    const C f0 = a0 < Q ? pull(a0) : C(0);
    const C f1 = a1 < Q ? pull(a1) : C(0);

    // moments (Eq. (3)), summed over the warp
    const C ex0 = a0 < Q ? C(s_ex[a0]) : C(0), ey0 = a0 < Q ? C(s_ey[a0]) : C(0);
    const C ex1 = a1 < Q ? C(s_ex[a1]) : C(0), ey1 = a1 < Q ? C(s_ey[a1]) : C(0);
    const C r0 = warp_allsum(f0 + f1);
    const C jx = warp_allsum(ex0 * f0 + ex1 * f1);
    const C jy = warp_allsum(ey0 * f0 + ey1 * f1);
    Collision<Q, C, SHIFT> col;
    const C drho = r0;
    col.rho = SHIFT ? C(1) + r0 : r0;
    const C inv = C(1) / col.rho;
    const C ux = k.r * jx * inv, uy = k.r * jy * inv;
    const C u2 = ux * ux + uy * uy;
    C th = 0, T = 1;
    if (k.thermal) {
        const C e2 = warp_allsum((ex0 * ex0 + ey0 * ey0) * f0 + (ex1 * ex1 + ey1 * ey1) * f1);
        if (SHIFT) {
            th = (k.th0 + k.r2 * e2 - col.rho * u2 - C(2) * drho) * (C(0.5) * inv);
            T = C(1) + th;
        } else {
            T = (k.r2 * e2 * inv - u2) * C(0.5);
            th = T - C(1);
        }
    }
    C taul;
    if (k.const_tau) taul = k.tau_lat;
    else if (k.mu_is_one || !k.thermal) taul = k.K * inv;
    else taul = k.K * inv * pow(T, k.mu_m1);
    const C om = C(1) / (taul + C(0.5));
    col.set_omega(om);
    col.sx = k.r * ux;
    col.sy = k.r * uy;
    // Eq. (4) coefficients: the c2-independent factors in every lane, those
    // of shell s in lane s only (the per-shell work is not repeated by every
    // lane, which matters where FP64 instructions are slow); each lane then
    // takes its velocities' shells' values by shuffle
    // (FP64 only: in FP32 the replicated per-shell work is cheaper than the
    // shuffles, measured)
    const int sh0 = a0 < Q ? s_sh[a0] : 0, sh1 = a1 < Q ? s_sh[a1] : 0;
    C A0v[2], A1v[2], A2v[2], cwv[2];
    if constexpr (sizeof(C) == 8) {
        C pw[8];
        col.powers(u2, th, drho * inv, k, pw);
        C sA0 = 0, sA1 = 0, sA2 = 0, scw = 0;
        if (lane < Lat<Q>::NSH)
            Collision<Q, C, SHIFT>::shell(pw, om * col.rho, k, lane, sA0, sA1, sA2, scw);
        const int shv[2] = {sh0, sh1};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            A0v[i] = __shfl_sync(0xffffffffu, sA0, shv[i]);
            A1v[i] = __shfl_sync(0xffffffffu, sA1, shv[i]);
            A2v[i] = __shfl_sync(0xffffffffu, sA2, shv[i]);
            cwv[i] = __shfl_sync(0xffffffffu, scw, shv[i]);
        }
    } else {
        col.set_coefficients(u2, th, om * col.rho, drho * inv, k);
        const int shv[2] = {sh0, sh1};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            A0v[i] = col.A0[shv[i]];
            A1v[i] = col.A1[shv[i]];
            A2v[i] = col.A2[shv[i]];
            cwv[i] = col.cw[shv[i]];
        }
    }

    // relax and store this lane's velocities (Eq. (4)-(5)); i: 0 for a0, 1 for a1
    auto relax_store = [&](int a, int i, C f) {
        const C sv = C(s_ex[a]) * col.sx + C(s_ey[a]) * col.sy;
        const C s2 = sv * sv;
        const C E = A0v[i] + s2 * (A2v[i] + col.A4 * s2);
        const C O = sv * (A1v[i] + col.A3 * s2);
        C v = col.relax(f, cwv[i] * (E + O));
        if constexpr (Store<PREC>::dev) v = f_to_dev(v, k.w[a], col.rho);
        store_pop<S>(fout, k, a, j, x, store_rounded<S>(v, sr_bits(hcell, a)));
    };
    if (a0 < Q) relax_store(a0, 0, f0);
    if (a1 < Q) relax_store(a1, 1, f1);
    if constexpr (Store<PREC>::dev)
        if (lane == 0) store_rho(rout, k, j, x, (float)col.rho);
}

}  // namespace lbm
