// Batched chunk kernel: many independent single-column Couette instances
// (Nx = 1, each with its own lattice, height, Kn, wall speeds and wall
// temperatures) advanced together, one CTA per slot, `chunk` time steps per
// launch, then an FP64 steady-state residual per slot.
//
// With Nx = 1 the pull of Eq. (5) only shifts in y: f_in(j, a) =
// f~*(j - e_ay, a).  Per step one warp sums the incoming mass of each wall
// (numerator of Eq. (12)): lane l loads the l-th (velocity, row) term of the
// wall's list (built on the host, carried in the slot descriptor), then a
// warp-shuffle FP64 reduction in a fixed lane order gives
// M_in; every slot's arithmetic is independent of the slot index, the grid
// and the other slots.
#pragma once

#include "batch_internal.h"
#include "lbm_device.cuh"

namespace lbm {

// Shared per-step wall data of a slot: the re-emitted deviations of Eq. (12)
// per wall and velocity, and the accommodation of each wall in FP32.
struct BatchWallShared {
    float fill[2][kMaxQ];
    float acc[2];
};

template <int Q>
__device__ __forceinline__ void batch_slot(const SlotDesc &d, float *__restrict__ pool,
                                           SlotStatus *__restrict__ st, BatchWallShared &sw) {
    const int chunk = d.chunk_steps;
    using L = Lat<Q>;
    const KConsts<float> &k = d.k;
    const int Ny = d.Ny;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int NT = d.nterm;                // <= 32, checked with the descriptor

    float *buf0 = pool + d.f_off;
    float *buf1 = buf0 + (long long)Q * Ny;
    const float *src = d.cur ? buf1 : buf0;
    float *dst = d.cur ? buf0 : buf1;

    if (tid < 2) sw.acc[tid] = (float)k.accom[tid];
    for (int step = 0; step < chunk; ++step) {
        if (warp < 2) {
            // numerator of Eq. (12) in FP64, then the normalised re-emission
            // M_in g^w_a / D_w of each outgoing velocity, formed in FP64 once
            // per wall and step (lane a and a + 32) and kept as an FP32
            // deviation: GB300's FP64 rate is a small fraction of its FP32 rate,
            // so no FP64 work is left in the per-cell loop
            double v = 0.0;
            if (lane < NT) {
                const int a = d.term_a[warp][lane];
                const int kk = d.term_row[warp][lane];
                const int row = warp == 0 ? kk : Ny - 1 - kk;
                // stored deviations: f = d + w
                v = (double)src[(long long)a * Ny + row] + (double)k.w[a];
            }
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            const double m = __shfl_sync(0xffffffffu, v, 0);
            for (int a = lane; a < Q; a += 32)
                sw.fill[warp][a] = k.wcoef[warp][a] != 0.0
                                       ? (float)(m * k.wcoef[warp][a] - (double)k.w[a]) : 0.0f;
        }
        __syncthreads();
        for (int j = tid; j < Ny; j += nth) {
            // the slot's constants live in shared memory; this compiler barrier
            // keeps them there (re-read per cell) instead of hoisted into
            // registers for the whole step loop, which spilled
            asm volatile("" ::: "memory");
            float f[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const int sj = j - L::ey(a);
                if (sj < 0 || sj >= Ny) {
                    // Eq. (9): diffuse part of the wall, plus the specular part
                    // (the mirrored velocity of the same row) when accom < 1;
                    // both are deviations from w_a, so the mix is linear in them
                    const int wall = sj < 0 ? 0 : 1;
                    const float acc = sw.acc[wall];
                    float v = sw.fill[wall][a];
                    if (acc != 1.0f)
                        v = acc * v + (1.0f - acc) * src[(long long)k.mirror[a] * Ny + j];
                    f[a] = v;
                } else {
                    f[a] = src[(long long)a * Ny + sj];
                }
            }
            Collision<Q, float, true> col;
            col.setup(f, k);
            float o[Q];
            o[0] = col.rest(f[0]);
            PairLoop<1, Q>::run([&](auto ic) {
                constexpr int A = decltype(ic)::value;
                col.template pair<A>(f[A], f[A + 1], o[A], o[A + 1]);
            });
#pragma unroll
            for (int a = 0; a < Q; ++a) dst[(long long)a * Ny + j] = o[a];
        }
        __syncthreads();
        const float *t = src;
        src = dst;
        dst = (float *)t;
    }

    const int chunks = st->chunks + 1;     // read before thread 0 updates it
    __syncthreads();
    if (tid == 0) st->chunks = chunks;
    if (chunks % d.check_every != 0) {
        if (tid == 0) {
            st->steps += chunk;
            if (st->steps >= d.max_steps) st->state = kSlotMaxSteps;
        }
        return;
    }

    // residual over the slot's cells (Eq. (3) moments of the current state)
    float *prev_u = (float *)(pool + d.prev_off);
    float *prev_T = prev_u + Ny;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const double r = (double)k.r;
    for (int j = tid; j < Ny; j += nth) {
        // deviations d = f - w: rho = 1 + sum d, sum e w = 0, sum e^2 w = e2w
        double s0 = 0, sx = 0, sy = 0, se = (double)k.e2w;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double fa = (double)src[(long long)a * Ny + j];
            s0 += fa;
            sx += L::ex(a) * fa;
            sy += L::ey(a) * fa;
            se += L::e2(a) * fa;
        }
        const double rh = 1.0 + s0;
        const double u = r * sx / rh, v = r * sy / rh;
        const double T = ((double)k.r2 * se - rh * (u * u + v * v)) / (2.0 * rh);
        const double du = u - prev_u[j], dT = T - prev_T[j];
        acc[0] += du * du;
        acc[1] += u * u;
        acc[2] += dT * dT;
        acc[3] += T * T;
        acc[4] += rh;
        if (!isfinite(u) || !isfinite(T)) acc[5] += 1.0;
        prev_u[j] = (float)u;
        prev_T[j] = (float)T;
    }
    __shared__ double red[32][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
        for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
    if (lane == 0)
        for (int i = 0; i < 6; ++i) red[warp][i] = acc[i];
    __syncthreads();
    if (tid == 0) {
        double tot[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < (nth + 31) / 32; ++w)
            for (int i = 0; i < 6; ++i) tot[i] += red[w][i];
        SlotStatus &s = *st;
        s.steps += chunk;
        s.checks += 1;
        s.mass = tot[4];
        double res = sqrt(tot[0]) / fmax(sqrt(tot[1]), 1e-30);
        if (k.thermal) res = fmax(res, sqrt(tot[2]) / fmax(sqrt(tot[3]), 1e-30));
        // geometric extrapolation of the remaining change: with a per-check
        // contraction q = res / res_prev < 1, the distance to the steady state
        // is about res q / (1 - q)
        // q from the last two checks, the slower of the two contractions
        const double q1 = s.res > 0 ? res / s.res : 1.0;
        const double q0 = s.res_prev > 0 ? s.res / s.res_prev : 1.0;
        const double q = fmax(q1, q0);
        const double prev_est = s.err_est;
        s.res_prev = s.res;
        s.res = res;
        s.err_est = (q < 0.999) ? res * q / (1.0 - q) : 1e30;
        if (res < s.best_res) { s.best_res = res; s.since_best = 0; }
        else s.since_best += 1;
        if (tot[5] > 0 || !isfinite(res)) s.state = kSlotNonFinite;
        else if (s.checks >= 4 && s.err_est <= d.tol && prev_est <= d.tol) s.state = kSlotConverged;
        // the residual stopped improving far below tol: the column has reached
        // the FP32 round-off floor (the check interval makes the slowest mode's
        // decay visible, so a flat, tiny residual is noise, not slow convergence)
        else if (s.since_best >= 8 && s.best_res <= 0.05 * d.tol) s.state = kSlotConverged;
        else if (s.since_best >= 50) s.state = kSlotStagnated;
        else if (s.steps >= d.max_steps) s.state = kSlotMaxSteps;
    }
}


}  // namespace lbm
