// Batched chunk kernel: many independent single-column Couette instances
// (Nx = 1, each with its own lattice, height, Kn, wall speeds and wall
// temperatures) advanced together, `chunk` time steps per launch, then an
// FP64 steady-state residual per slot.
//
// With Nx = 1 the pull of Eq. (5) only shifts in y: f_in(j, a) =
// f~*(j - e_ay, a).  A slot runs on a cluster of CL CTAs (CL = 1, 2, 4 or 8,
// fixed by its height): CTA `rank` owns rows [rank R, rank R + R), R =
// ceil(Ny / CL), and a cluster barrier with release / acquire semantics
// separates the steps.  When R <= kSmemRows the CTA keeps its rows' two state
// buffers in shared memory for the whole chunk (loaded from the pool at the
// start, written back at the end) and pulls the <= 3 rows it needs from each
// neighbour through distributed shared memory; taller slots keep the state in
// global memory (L2-resident) and read it with ld.global.cg.
//
// Row mapping inside a CTA: warp 0 of the bottom CTA owns the (up to) 32
// lowest rows and warp 1 of the top CTA the 32 highest; each of those warps
// first sums its wall's incoming mass (numerator of Eq. (12)) in FP64 by a
// warp shuffle in a fixed lane order - lane l loads the l-th (velocity, row)
// term of the wall's list, built on the host and carried in the slot
// descriptor - forms the normalised re-emission of every outgoing velocity
// once, and then updates its rows.  The other rows never need a wall value,
// so no block barrier separates the wall sums from the bulk update.  Every
// slot's arithmetic depends only on the slot itself (its cluster size is a
// function of its height), never on the slot index, the grid or other slots.
#pragma once

#include "batch_internal.h"
#include "lbm_device.cuh"

namespace lbm {

// Shared per-step wall data of a slot: the re-emitted deviations of Eq. (12)
// per wall and velocity and the accommodation of each wall in FP32, plus the
// block-reduction scratch of the residual.
struct BatchWallShared {
    float fill[2][kMaxQ];
    float acc[2];
    double red[32][6];
};

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}

// Barrier of all threads of the slot's cluster, with release / acquire
// semantics at cluster scope: every global store of the cluster before it is
// visible to every thread of the cluster after it.  One CTA: the block barrier.
__device__ __forceinline__ void slot_barrier(int CL) {
    if (CL == 1) {
        __syncthreads();
        return;
    }
    // non-.aligned forms: correct even if a warp arrives diverged
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}

// Rows of a CTA's shared-memory state: two buffers of Q x kSmemRows floats.
constexpr int kSmemRows = 256;
constexpr int kSmemBytes = 2 * kMaxQ * kSmemRows * (int)sizeof(float);

// Generic address of the same shared-memory location in CTA `rank` of the
// cluster (distributed shared memory).
__device__ __forceinline__ float *map_rank(float *p, unsigned rank) {
    unsigned long long out;
    asm volatile("mapa.u64 %0, %1, %2;\n" : "=l"(out) : "l"((unsigned long long)p), "r"(rank));
    return (float *)out;
}

// Slot state in global memory (pool), two buffers of [Q][Ny]; a step reads
// `src` and writes `dst`, rows of any CTA of the cluster.
struct GlobalState {
    const float *src;
    float *dst;
    int Ny;
    // population a of slot row `row` of the current state (coherent L2 read:
    // another SM may have written it)
    __device__ __forceinline__ float ld(int a, int row) const {
        return __ldcg(src + (long long)a * Ny + row);
    }
    __device__ __forceinline__ float ld_own(int a, int row) const { return ld(a, row); }
    __device__ __forceinline__ void st(int a, int row, float v) const {
        dst[(long long)a * Ny + row] = v;
    }
    __device__ __forceinline__ void flip() {
        const float *t = src;
        src = dst;
        dst = (float *)t;
    }
};

// Slot state in the cluster's shared memory: this CTA holds rows [j0, j0 + R)
// as buf[b][a][row - j0] (b = current buffer); lo / hi are the same buffers of
// the neighbouring CTAs (rows j0 - R .., j0 + R ..), null at the slot's ends.
struct SmemState {
    float *buf;                // local buffers, 2 x Q x R floats
    const float *lo, *hi;      // neighbours' buffers (distributed shared memory)
    int R, j0, QR, b;
    __device__ __forceinline__ float ld(int a, int row) const {
        int lr = row - j0;
        const float *p = buf;
        if (lr < 0) {
            p = lo;
            lr += R;
        } else if (lr >= R) {
            p = hi;
            lr -= R;
        }
        return p[b * QR + a * R + lr];
    }
    __device__ __forceinline__ float ld_own(int a, int row) const {
        return buf[b * QR + a * R + row - j0];
    }
    __device__ __forceinline__ void st(int a, int row, float v) const {
        buf[(b ^ 1) * QR + a * R + row - j0] = v;
    }
    __device__ __forceinline__ void flip() { b ^= 1; }
};

// Numerator of Eq. (12) for `wall` summed by one full warp in FP64, and the
// normalised re-emission M_in g^w_a / D_w of each outgoing velocity formed
// once in FP64 (lanes a and a + 32) and kept as an FP32 deviation from w_a:
// GB300's FP64 rate is a small fraction of its FP32 rate, so no FP64 work is
// left in the per-cell update.  The wall rows belong to this CTA.
template <int Q, class State>
__device__ __forceinline__ void wall_fill_warp(const SlotDesc &d, const State &S, int wall,
                                               int lane, float *fill) {
    const KConsts<float> &k = d.k;
    double v = 0.0;
    if (lane < d.nterm) {
        const int a = d.term_a[wall][lane];
        const int kk = d.term_row[wall][lane];
        const int row = wall == 0 ? kk : d.Ny - 1 - kk;
        v = (double)S.ld_own(a, row) + (double)k.w[a];   // f = d + w
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const double m = __shfl_sync(0xffffffffu, v, 0);
    for (int a = lane; a < Q; a += 32)
        fill[a] = k.wcoef[wall][a] != 0.0 ? (float)(m * k.wcoef[wall][a] - (double)k.w[a]) : 0.0f;
    __syncwarp();
}

// Pull, collide and store row j (Eq. (5) with the Eq. (9)-(12) wall).  EDGE:
// the row is within 3 rows of its CTA's first or last row, so a source may lie
// beyond the slot's walls or in a neighbouring CTA; otherwise every source is
// one of this CTA's rows.
template <int Q, bool EDGE, class State>
__device__ __forceinline__ void cell_update(const SlotDesc &d, const State &S, int j,
                                            const BatchWallShared &sw) {
    using L = Lat<Q>;
    // the slot's constants live in shared memory; this compiler barrier keeps
    // them there (re-read per cell) instead of hoisted into registers for the
    // whole step loop, which spilled
    asm volatile("" ::: "memory");
    const KConsts<float> &k = d.k;
    const int Ny = d.Ny;
    float f[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int sj = j - L::ey(a);
        if (!EDGE) {
            f[a] = S.ld_own(a, sj);
        } else if (sj < 0 || sj >= Ny) {
            // Eq. (9): diffuse part of the wall, plus the specular part (the
            // mirrored velocity of the same row) when accom < 1; both are
            // deviations from w_a, so the mix is linear in them
            const int wall = sj < 0 ? 0 : 1;
            const float acc = sw.acc[wall];
            float v = sw.fill[wall][a];
            if (acc != 1.0f) v = acc * v + (1.0f - acc) * S.ld_own(k.mirror[a], j);
            f[a] = v;
        } else {
            f[a] = S.ld(a, sj);
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
    for (int a = 0; a < Q; ++a) S.st(a, j, o[a]);
}

// The chunk's time steps.  Warp 0 of the bottom CTA and warp 1 of the top CTA
// own the wall blocks [j0, j0 + nb) and [j1 - nt, j1) and first form their
// wall's re-emission; every thread then updates its wall-block row (if any)
// and its share of the bulk rows [mb, me), handed out from the last thread
// down so that the wall warps get bulk rows last.
template <int Q, class State>
__device__ __forceinline__ void run_steps(const SlotDesc &d, State &S, BatchWallShared &sw,
                                          int chunk, int CL, int warp, int lane, int tid,
                                          int nth, int j0, int j1, int nb, int nt, int mb,
                                          int me) {
    int jw = -1;
    if (warp == 0 && nb > 0 && lane < nb) jw = j0 + lane;
    if (warp == 1 && nt > 0 && lane < nt) jw = j1 - nt + lane;
    const int jb = mb + (nth - 1 - tid);
    for (int step = 0; step < chunk; ++step) {
        if (warp == 0 && nb > 0) wall_fill_warp<Q>(d, S, 0, lane, sw.fill[0]);
        else if (warp == 1 && nt > 0) wall_fill_warp<Q>(d, S, 1, lane, sw.fill[1]);
        for (int it = jw >= 0 ? -1 : 0;; ++it) {
            const int j = it < 0 ? jw : jb + it * nth;
            if (it >= 0 && j >= me) break;
            if (j < j0 + 3 || j >= j1 - 3) cell_update<Q, true>(d, S, j, sw);
            else cell_update<Q, false>(d, S, j, sw);
        }
        slot_barrier(CL);
        S.flip();
    }
}

// One chunk of one slot on CTA `rank` of its CL-CTA cluster.  `chunks` is the
// slot's chunk counter after this chunk (read by every CTA before the first
// barrier); `part` holds CL x 6 FP64 partial sums of the residual; `sm` the
// CTA's kSmemBytes of dynamic shared memory (used when R <= kSmemRows).
template <int Q>
__device__ __forceinline__ void batch_slot(const SlotDesc &d, float *__restrict__ pool,
                                           SlotStatus *__restrict__ st, BatchWallShared &sw,
                                           int rank, int CL, int chunks,
                                           double *__restrict__ part, float *sm) {
    using L = Lat<Q>;
    const int chunk = d.chunk_steps;
    const KConsts<float> &k = d.k;
    const int Ny = d.Ny;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int R = (Ny + CL - 1) / CL;
    const int j0 = min(Ny, rank * R), j1 = min(Ny, j0 + R);
    const bool has_bot = rank == 0, has_top = rank == CL - 1;
    const int span = j1 - j0;
    // wall blocks: >= 3 rows each (every row that pulls from a wall), since
    // the host keeps Ny >= 6 and R >= 32 whenever CL > 1
    int nb = 0, nt = 0;
    if (has_bot && has_top) {
        nb = min(32, span / 2);
        nt = min(32, span - nb);
    } else if (has_bot) {
        nb = min(32, span);
    } else if (has_top) {
        nt = min(32, span);
    }
    const int mb = j0 + nb, me = j1 - nt;

    float *g_cur = pool + d.f_off + (d.cur ? (long long)Q * Ny : 0);
    float *g_oth = pool + d.f_off + (d.cur ? 0 : (long long)Q * Ny);
    const bool smem = R <= kSmemRows;
    const float *fin;                          // the state after the chunk
    if (tid < 2) sw.acc[tid] = (float)k.accom[tid];
    if (smem) {
        // own rows into buffer 0
        for (int i = tid; i < Q * span; i += nth) {
            const int a = i / span, r = i - a * span;
            sm[a * R + r] = __ldcg(g_cur + (long long)a * Ny + j0 + r);
        }
        SmemState S{sm, nullptr, nullptr, R, j0, Q * R, 0};
        if (rank > 0) S.lo = map_rank(sm, rank - 1);
        if (rank < CL - 1) S.hi = map_rank(sm, rank + 1);
        slot_barrier(CL);                      // every CTA loaded before any neighbour reads
        run_steps<Q>(d, S, sw, chunk, CL, warp, lane, tid, nth, j0, j1, nb, nt, mb, me);
        fin = sm + S.b * Q * R;
        // write the final state back to the pool buffer it came from
        for (int i = tid; i < Q * span; i += nth) {
            const int a = i / span, r = i - a * span;
            g_cur[(long long)a * Ny + j0 + r] = fin[a * R + r];
        }
    } else {
        __syncthreads();
        GlobalState S{g_cur, g_oth, Ny};
        run_steps<Q>(d, S, sw, chunk, CL, warp, lane, tid, nth, j0, j1, nb, nt, mb, me);
        fin = S.src;
    }

    if (chunks % d.check_every != 0) {
        if (rank == 0 && tid == 0) {
            st->chunks = chunks;
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
    for (int j = j0 + tid; j < j1; j += nth) {
        // deviations d = f - w: rho = 1 + sum d, sum e w = 0, sum e^2 w = e2w
        double s0 = 0, sx = 0, sy = 0, se = (double)k.e2w;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double fa = smem ? (double)fin[a * R + j - j0]
                                   : (double)__ldcg(fin + (long long)a * Ny + j);
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
#pragma unroll
    for (int i = 0; i < 6; ++i)
        for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
    if (lane == 0)
        for (int i = 0; i < 6; ++i) sw.red[warp][i] = acc[i];
    __syncthreads();
    double tot[6] = {0, 0, 0, 0, 0, 0};
    if (tid == 0)
        for (int w = 0; w < (nth + 31) / 32; ++w)
            for (int i = 0; i < 6; ++i) tot[i] += sw.red[w][i];
    if (CL > 1) {
        // CTA partials through global memory, summed by rank 0 in rank order
        if (tid == 0)
            for (int i = 0; i < 6; ++i) part[rank * 6 + i] = tot[i];
        slot_barrier(CL);
        if (rank != 0) return;
        if (tid == 0)
            for (int i = 0; i < 6; ++i) {
                tot[i] = 0.0;
                for (int c = 0; c < CL; ++c) tot[i] += part[c * 6 + i];
            }
    }
    if (tid == 0) {
        SlotStatus &s = *st;
        s.chunks = chunks;
        s.steps += chunk;
        s.checks += 1;
        s.mass = tot[4];
        double res = sqrt(tot[0]) / fmax(sqrt(tot[1]), 1e-30);
        if (k.thermal) res = fmax(res, sqrt(tot[2]) / fmax(sqrt(tot[3]), 1e-30));
        // geometric extrapolation of the remaining change: with a per-check
        // contraction q = res / res_prev < 1, the distance to the steady state
        // is about res q / (1 - q); q from the last two checks, the slower of
        // the two contractions
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
