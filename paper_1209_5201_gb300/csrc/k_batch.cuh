// Batched chunk kernel: many independent single-column Couette instances
// (Nx = 1, each with its own lattice, height, Kn, wall speeds and wall
// temperatures) advanced together, `sub` chunks of `chunk` time steps per
// launch, with an FP64 steady-state residual after every check_every-th
// chunk of a slot.
//
// With Nx = 1 the pull of Eq. (5) only shifts in y: f_in(j, a) =
// f~*(j - e_ay, a).  A slot runs on a cluster of CL CTAs (CL = 1, 2, 4, 8 or
// 16, fixed by its height): CTA `rank` owns rows [rank R, rank R + R), R =
// ceil(Ny / CL), and a cluster barrier with release / acquire semantics
// separates the steps.  When R <= kSmemRows the CTA keeps its rows' two state
// buffers in shared memory for the whole launch (loaded from the pool at the
// start, written back at the end; rows of Q populations) and pulls the <= 3
// rows it needs from each neighbour through distributed shared memory
// (ld.shared::cluster); taller blocks keep the state in global memory
// (L2-resident) and read it with ld.global.cg.
//
// Row mapping inside a CTA: warp 0 of the bottom CTA owns the (up to) 32
// lowest rows and warp 1 of the top CTA the 32 highest; each of those warps
// first sums its wall's incoming mass (numerator of Eq. (12)) in FP64 by a
// warp shuffle in a fixed lane order - lane l loads the l-th (velocity, row)
// term of the wall's list, built on the host and carried in the slot
// descriptor - forms the normalised re-emission of every outgoing velocity
// once, and then updates its rows (branch-free: sources clamped into the
// slot, the wall's values selected afterwards).  The other rows never need a wall value,
// so no block barrier separates the wall sums from the bulk update.  Every
// slot's arithmetic depends only on the slot itself (its cluster size is a
// function of its height), never on the slot index, the grid or other slots.
#pragma once

#include "batch_internal.h"
#include "lbm_device.cuh"

namespace lbm {

// Shared per-step wall data of a slot: the re-emitted deviations of Eq. (12)
// per wall and velocity, the accommodation of each wall in FP32, and (state in
// global memory) the post-collision values of the 3 rows next to each wall,
// term[w][kk][a] at distance kk from wall w, which the next step's wall sum
// reads from here instead of from L2.
struct BatchWallShared {
    float fill[2][kMaxQ];
    float acc[2];
    float term[2][3][kMaxQ];
};

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}

// Barrier of all threads of the slot's cluster, with release / acquire
// semantics at cluster scope: every global store of the cluster before it is
// visible to every thread of the cluster after it.  One CTA: the block barrier.
__device__ __forceinline__ void cluster_arrive() {
    // non-.aligned forms: correct even if a warp arrives diverged
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}
__device__ __forceinline__ void slot_barrier(int CL) {
    if (CL == 1) {
        __syncthreads();
        return;
    }
    cluster_arrive();
    cluster_wait();
}

// Rows of a CTA's shared-memory state: two buffers of Q x kSmemRows floats.
constexpr int kSmemRows = 256;
constexpr int kSmemBytes = 2 * kMaxQ * kSmemRows * (int)sizeof(float);

// The shared-memory path serves every column whose CTAs' rows fit.
__host__ __device__ inline bool batch_uses_smem(int Ny, int CL) {
    return batch_rows_per_cta(Ny, CL) <= kSmemRows;
}

// Population a of the wall re-emission (Eq. (9) with R = accom R_D + (1 -
// accom) R_S): the diffuse part formed by the wall warp, plus the specular
// part (the mirrored velocity of the same row, `spec`, read only when accom <
// 1); both are deviations from w_a, so the mix is linear in them.
template <class SpecFn>
__device__ __forceinline__ float wall_value(const BatchWallShared &sw, int wall, int a,
                                            SpecFn &&spec) {
    const float acc = sw.acc[wall];
    float v = sw.fill[wall][a];
    if (acc != 1.0f) v = acc * v + (1.0f - acc) * spec();
    return v;
}

// Wall rows of a pull (EDGE): f[a] was loaded from the source row clamped into
// the slot; where the true source lies beyond a wall (e_y > j bottom, j - e_y
// >= Ny top) it is replaced by that wall's re-emission.  Without specular
// reflection the replacement is a predicated select, so the pull has no
// branch between its loads.
template <int Q, class MirrorFn>
__device__ __forceinline__ void apply_walls(const BatchWallShared &sw, int j, int Ny,
                                            float (&f)[Q], MirrorFn &&mirror) {
    using L = Lat<Q>;
    if (sw.acc[0] == 1.0f && sw.acc[1] == 1.0f) {
        StaticFor<0, Q>::run([&](auto ic) {
            constexpr int a = decltype(ic)::value;
            if constexpr (L::ey(a) > 0) f[a] = j - L::ey(a) < 0 ? sw.fill[0][a] : f[a];
            else if constexpr (L::ey(a) < 0) f[a] = j - L::ey(a) >= Ny ? sw.fill[1][a] : f[a];
        });
    } else {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int sj = j - L::ey(a);
            if (sj < 0 || sj >= Ny)
                f[a] = wall_value(sw, sj < 0 ? 0 : 1, a, [&] { return mirror(a); });
        }
    }
}

// Slot state in global memory (pool), two buffers of [Q][Ny]; a step reads
// `src` and writes `dst`, rows of any CTA of the cluster.
struct GlobalState {
    const float *src;
    float *dst;
    int Ny;
    float *stage;              // BatchWallShared::term of this CTA
    // population a of slot row `row` of the current state (coherent L2 read:
    // another SM may have written it)
    __device__ __forceinline__ float ld(int a, int row) const {
        return __ldcg(src + (long long)a * Ny + row);
    }
    __device__ __forceinline__ float ld_own(int a, int row) const { return ld(a, row); }
    // wall w's incoming term (a, kk) of the step just done (staged by store)
    __device__ __forceinline__ float term(int w, int a, int kk, int) const {
        return stage[(w * 3 + kk) * kMaxQ + a];
    }
    // f_in of row j (Eq. (5) pull with the Eq. (12) wall)
    template <int Q, bool EDGE>
    __device__ __forceinline__ void pull(const SlotDesc &d, const BatchWallShared &sw, int j,
                                         float (&f)[Q]) const {
        using L = Lat<Q>;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int sj = j - L::ey(a);
            f[a] = ld(a, EDGE ? min(max(sj, 0), Ny - 1) : sj);
        }
        if constexpr (EDGE) apply_walls<Q>(sw, j, Ny, f, [&](int a) { return ld(d.k.mirror[a], j); });
    }
    template <int Q, bool EDGE>
    __device__ __forceinline__ void store(int j, const float (&o)[Q]) const {
        using L = Lat<Q>;
#pragma unroll
        for (int a = 0; a < Q; ++a) dst[(long long)a * Ny + j] = o[a];
        if constexpr (EDGE) {
            // the velocities that stream into a wall from its 3 nearest rows
            if (j < 3) {
                StaticFor<0, Q>::run([&](auto ic) {
                    constexpr int a = decltype(ic)::value;
                    if constexpr (L::ey(a) < 0) stage[j * kMaxQ + a] = o[a];
                });
            } else if (j >= Ny - 3) {
                StaticFor<0, Q>::run([&](auto ic) {
                    constexpr int a = decltype(ic)::value;
                    if constexpr (L::ey(a) > 0) stage[(3 + Ny - 1 - j) * kMaxQ + a] = o[a];
                });
            }
        }
    }
    __device__ __forceinline__ void flip() {
        const float *t = src;
        src = dst;
        dst = (float *)t;
    }
};

__device__ __forceinline__ float lds_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(addr) : "memory");
    return v;
}
template <int OFF>
__device__ __forceinline__ float lds_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];\n" : "=f"(v) : "r"(addr), "n"(OFF) : "memory");
    return v;
}
template <int OFF>
__device__ __forceinline__ void sts_f32(uint32_t addr, float v) {
    asm volatile("st.shared.f32 [%0+%1], %2;\n" ::"r"(addr), "n"(OFF), "f"(v) : "memory");
}
// Load through the shared::cluster window (this CTA's or a neighbour's
// shared memory), without a compiler memory clobber: ordered only against the
// other volatile asm (the loads, stores and barriers of this file), so the
// constants read around it can stay in registers.
__device__ __forceinline__ float ldsc_f32_nc(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];\n" : "=f"(v) : "r"(addr));
    return v;
}
// shared::cluster address of the same location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, unsigned rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(out) : "r"(addr), "r"(rank));
    return out;
}

// Slot state in the cluster's shared memory.  This CTA holds rows [j0, j0 + R)
// in two buffers of R rows x Q floats (row-major: a thread's Q populations are
// contiguous and Q is odd, so the 32 lanes of a warp, on 32 consecutive rows,
// hit 32 different banks); `b` is the buffer holding the current state.  lo /
// hi are the same buffers of the neighbouring CTAs (rows j0 - R .., j0 + R ..)
// as shared::cluster addresses, 0 at the slot's ends.  Bulk rows read with
// compile-time offsets from their own row address.
template <int Q>
struct SmemState {
    uint32_t base;             // shared::cta address of buffer 0
    uint32_t lo, hi;           // shared::cluster addresses of the neighbours' buffer 0
    uint32_t self;             // shared::cluster address of this CTA's buffer 0
    int R, j0, b;
    __device__ __forceinline__ uint32_t row_addr(int buf, int lr) const {
        return base + (uint32_t)((buf * R + lr) * Q) * 4u;
    }
    __device__ __forceinline__ float ld_own(int a, int row) const {
        return lds_f32(row_addr(b, row - j0) + (uint32_t)a * 4u);
    }
    // wall w's incoming term (a, kk): row kk from the wall of the current state
    __device__ __forceinline__ float term(int w, int a, int kk, int Ny) const {
        return ld_own(a, w == 0 ? kk : Ny - 1 - kk);
    }
    template <int Q_, bool EDGE>
    __device__ __forceinline__ void pull(const SlotDesc &d, const BatchWallShared &sw, int j,
                                         float (&f)[Q_]) const {
        using L = Lat<Q_>;
        if constexpr (!EDGE) {
            // every source row lies in [lr - 3, lr + 3] of this CTA: offsets
            // from row lr - 3 are compile-time constants
            const uint32_t r0 = row_addr(b, j - j0 - 3);
            StaticFor<0, Q_>::run([&](auto ic) {
                constexpr int a = decltype(ic)::value;
                f[a] = lds_f32<((3 - L::ey(a)) * Q_ + a) * 4>(r0);
            });
        } else {
            // source row clamped into the slot, then into this CTA or a
            // neighbour (selects, no branch): every load goes through the
            // shared::cluster window and all of them issue back to back
#pragma unroll
            for (int a = 0; a < Q_; ++a) {
                const int lr = min(max(j - L::ey(a), 0), d.Ny - 1) - j0;
                const uint32_t bse = lr < 0 ? lo : (lr >= R ? hi : self);
                const int rr = lr < 0 ? lr + R : (lr >= R ? lr - R : lr);
                f[a] = ldsc_f32_nc(bse + (uint32_t)(((b * R + rr) * Q_ + a) * 4));
            }
            apply_walls<Q_>(sw, j, d.Ny, f, [&](int a) { return ld_own(d.k.mirror[a], j); });
        }
    }
    template <int Q_, bool EDGE>
    __device__ __forceinline__ void store(int j, const float (&o)[Q_]) const {
        const uint32_t r = row_addr(b ^ 1, j - j0);
        StaticFor<0, Q_>::run([&](auto ic) {
            constexpr int a = decltype(ic)::value;
            sts_f32<a * 4>(r, o[a]);
        });
    }
    __device__ __forceinline__ void flip() { b ^= 1; }
};

// Numerator of Eq. (12) for `wall` summed by one full warp in FP64, and the
// normalised re-emission M_in g^w_a / D_w of each outgoing velocity formed
// once in FP64 (lane l: outgoing velocity out_a[l]) and kept as an FP32
// deviation from w_a.  Lane l < nterm carries its term's deviation d = f - w,
// lane nterm the terms' weights summed on the host, so M_in = sum d + sum w;
// a butterfly of shuffles leaves the same fixed-order sum in every lane.
// GB300's FP64 rate is a small fraction of its FP32 rate: eight FP64
// instructions per wall and step, none in the per-cell update.  `term(a, kk)`
// reads the incoming term (a, kk) of the current state; the wall rows belong
// to this CTA.
// The FP32 value of each re-emission is rounded stochastically (add_sr of
// its round-to-nearest value and the FP32 remainder), from the hash of the
// step and a counter beyond the slot's rows.
template <class TermFn>
__device__ __forceinline__ void wall_fill_warp(const SlotDesc &d, int wall, int lane,
                                               float *fill, uint32_t step, TermFn &&term) {
    double v = 0.0;
    if (lane < d.nterm) v = (double)term(d.term_a[wall][lane], d.term_row[wall][lane]);
    else if (lane == d.nterm) v = d.wterm[wall];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane < d.nout) {
        const double x = fma(v, d.out_c[wall][lane], -d.out_w[wall][lane]);
        const float hi = (float)x, lo = (float)(x - (double)hi);
        const uint32_t h = sr_cell(step, (uint32_t)(d.Ny + wall));
        fill[d.out_a[wall][lane]] = add_sr(hi, lo, sr_bits32(h, lane));
    }
    __syncwarp();
}

// Pull, collide and store row j (Eq. (5) with the Eq. (9)-(12) wall).  EDGE:
// the row is within 3 rows of its CTA's first or last row, so a source may lie
// beyond the slot's walls or in a neighbouring CTA; otherwise every source is
// one of this CTA's rows.
// PRECISE: conserving increments with stochastic rounding (the steady-state
// phase of a solve); otherwise the plain relaxation rounded to nearest.
template <int Q, bool EDGE, bool PRECISE, class State>
__device__ __forceinline__ void cell_update(const SlotDesc &d, const State &S, int j,
                                            const BatchWallShared &sw, uint32_t step) {
    // the slot's constants live in shared memory; this compiler barrier keeps
    // them there (re-read per cell) instead of hoisted into registers for the
    // whole step loop, which spilled
    asm volatile("" ::: "memory");
    const KConsts<float> &k = d.k;
    float f[Q];
    S.template pull<Q, EDGE>(d, sw, j, f);
    Collision<Q, float, true> col;
    col.setup(f, k);
    // PRECISE: increments that conserve mass, momentum (and energy) in FP32,
    // added with stochastic rounding: random bits from the hash of the
    // request's step count and the row (the same however the column is split
    // or batched)
    float o[Q];
    if constexpr (PRECISE) {
        col.relax_conserving_sr(f, o, sr_cell(step, (uint32_t)j), k.thermal != 0);
    } else {
        o[0] = col.rest(f[0]);
        PairLoop<1, Q>::run([&](auto ic) {
            constexpr int A = decltype(ic)::value;
            col.template pair<A>(f[A], f[A + 1], o[A], o[A + 1]);
        });
    }
    S.template store<Q, EDGE>(j, o);
}

// The chunk's time steps.  Warp 0 of the bottom CTA and warp 1 of the top CTA
// own the wall blocks [j0, j0 + nb) and [j1 - nt, j1) and first form their
// wall's re-emission; every thread then updates its wall-block row (if any)
// and its share of the bulk rows [mb, me), handed out from the last thread
// down so that the wall warps get bulk rows last.
template <int Q, bool PRECISE, class State>
__device__ __forceinline__ void run_steps(const SlotDesc &d, State &S, BatchWallShared &sw,
                                          int chunk, int CL, int warp, int lane, int tid,
                                          int nth, int j0, int j1, int nb, int nt, int mb,
                                          int me, uint32_t step0) {
    int jw = -1;
    if (warp == 0 && nb > 0 && lane < nb) jw = j0 + lane;
    if (warp == 1 && nt > 0 && lane < nt) jw = j1 - nt + lane;
    const int jb = mb + (nth - 1 - tid);
    // a wall warp's incoming terms are rows of its own wall block
    const bool wall_warp = (warp == 0 && nb > 0) || (warp == 1 && nt > 0);
    const int wall = warp == 0 ? 0 : 1;
    const int Ny = d.Ny;
    // the chunk's first wall sums read the state as loaded; later ones the
    // wall rows just written (staged in shared memory on the global path)
    if (wall_warp)
        wall_fill_warp(d, wall, lane, sw.fill[wall], step0,
                       [&](int a, int kk) { return S.ld_own(a, wall == 0 ? kk : Ny - 1 - kk); });
    auto fill_next = [&](uint32_t st) {
        wall_fill_warp(d, wall, lane, sw.fill[wall], st,
                       [&](int a, int kk) { return S.term(wall, a, kk, Ny); });
    };
    for (int step = 0; step < chunk; ++step) {
        const uint32_t gstep = step0 + (uint32_t)step;
        for (int it = jw >= 0 ? -1 : 0;; ++it) {
            const int j = it < 0 ? jw : jb + it * nth;
            if (it >= 0 && j >= me) break;
            // one path per warp: a warp with any row within 3 rows of its
            // CTA's ends takes the general (EDGE) path for all its rows, so
            // the collision is never executed twice by a diverged warp
            const bool edge = __any_sync(__activemask(), j < j0 + 3 || j >= j1 - 3);
            if (edge) cell_update<Q, true, PRECISE>(d, S, j, sw, gstep);
            else cell_update<Q, false, PRECISE>(d, S, j, sw, gstep);
        }
        const bool more = step + 1 < chunk;
        if (CL == 1) {
            __syncthreads();
            S.flip();
            if (wall_warp && more) fill_next(gstep + 1u);
        } else {
            // the next step's wall sums read only rows this warp has just
            // written (visible to it after __syncwarp), so they run between
            // arriving at the cluster barrier and waiting on it
            cluster_arrive();
            S.flip();
            if (wall_warp && more) fill_next(gstep + 1u);
            cluster_wait();
        }
    }
}

// Up to d.sub chunks of one slot on CTA `rank` of its CL-CTA cluster
// (fewer when the slot stops: converged, stagnated, non-finite or at
// max_steps); returns the chunks run.  chunks0 / steps0 are the slot's
// counters before the launch (read by every CTA before the first barrier);
// `part` the slot's per-chunk FP64 partial sums of the residual; `sm` the
// CTA's kSmemBytes of dynamic shared memory (used when R <= kSmemRows).  A
// residual check follows every check_every-th chunk of the slot's count, so
// the checks fall on the same steps whatever the number of chunks per launch.
template <int Q>
__device__ __forceinline__ int batch_slot(const SlotDesc &d, float *__restrict__ pool,
                                          SlotStatus *__restrict__ st, BatchWallShared &sw,
                                          int rank, int CL, int chunks0, long long steps0,
                                          int precise, double *__restrict__ part, float *sm) {
    using L = Lat<Q>;
    const int chunk = d.chunk_steps;
    const KConsts<float> &k = d.k;
    const int Ny = d.Ny;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int R = batch_rows_per_cta(Ny, CL);
    const int j0 = min(Ny, rank * R), j1 = min(Ny, j0 + R);
    const bool has_bot = rank == 0, has_top = rank == CL - 1;
    const int span = j1 - j0;
    // wall blocks: >= 3 rows each (every row that pulls from a wall), since
    // the host keeps Ny >= 6 and every CTA of a split >= 32 rows
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
    const bool smem = batch_uses_smem(Ny, CL);

    // Change of the macroscopic fields since the last check (Eq. (3) moments
    // of the state `fin` after chunk ck), in the units of the accuracy the
    // solve is asked for: over the 32-row blocks of the column, the largest
    // change of a block's mean u_x divided by the wall speed u_ref, and for a
    // thermal lattice also the largest change of a block's mean T.  The block
    // means follow the smooth, slowly decaying modes that set the distance to
    // the steady state and average out the zero-mean noise of the stochastic
    // rounding.  Per 32-row block (one warp each) the changes, the mass and a
    // non-finite flag go to global memory, then one warp of CTA 0 combines
    // the blocks in a fixed order: the result does not depend on how the rows
    // were split across CTAs.  Returns whether the slot keeps running (the
    // same answer in every thread of the cluster).
    auto check = [&](const float *fin, int ck, long long steps_k) -> bool {
        float *prev_u = (float *)(pool + d.prev_off);
        float *prev_T = prev_u + Ny;
        const double r = (double)k.r;
        const int nwarps = nth >> 5;
        for (int c = j0 / kResidualChunk + warp; c * kResidualChunk < j1; c += nwarps) {
            const int j = c * kResidualChunk + lane;
            double acc[6] = {0, 0, 0, 0, 0, 0};
            if (j < j1) {
                // deviations d = f - w: rho = 1 + sum d, sum e w = 0, sum e^2 w = e2w
                double s0 = 0, sx = 0, sy = 0, se = (double)k.e2w;
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    const double fa = smem ? (double)fin[(j - j0) * Q + a]
                                           : (double)__ldcg(fin + (long long)a * Ny + j);
                    s0 += fa;
                    sx += L::ex(a) * fa;
                    sy += L::ey(a) * fa;
                    se += L::e2(a) * fa;
                }
                const double rh = 1.0 + s0;
                const double u = r * sx / rh, v = r * sy / rh;
                const double T = ((double)k.r2 * se - rh * (u * u + v * v)) / (2.0 * rh);
                const float uf = (float)u, Tf = (float)T;
                acc[0] = (double)uf - (double)prev_u[j];
                acc[2] = (double)Tf - (double)prev_T[j];
                acc[4] = rh;
                acc[5] = (!isfinite(u) || !isfinite(T)) ? 1.0 : 0.0;
                prev_u[j] = uf;
                prev_T[j] = Tf;
            }
#pragma unroll
            for (int i = 0; i < 6; ++i)
                for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
            if (lane == 0) {
                // block means of the changes (the block's rows: whole blocks
                // except at the top of the column)
                const double nrow = (double)min(kResidualChunk, Ny - c * kResidualChunk);
                acc[0] = fabs(acc[0]) / nrow;
                acc[2] = fabs(acc[2]) / nrow;
                for (int i = 0; i < 6; ++i) part[c * 6 + i] = acc[i];
            }
        }
        slot_barrier(CL);                      // every chunk's partials written
        if (rank == 0) {
            double tot[6] = {0, 0, 0, 0, 0, 0};
            if (warp == 0) {
                const int nch = (Ny + kResidualChunk - 1) / kResidualChunk;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const bool mx = i == 0 || i == 2;
                    double v = 0.0;
                    for (int c = lane; c < nch; c += 32) v = mx ? fmax(v, part[c * 6 + i]) : v + part[c * 6 + i];
                    for (int o = 16; o > 0; o >>= 1) {
                        const double x = __shfl_down_sync(0xffffffffu, v, o);
                        v = mx ? fmax(v, x) : v + x;
                    }
                    tot[i] = v;
                }
            }
            if (tid == 0) {
                SlotStatus &s = *st;
                s.chunks = ck;
                s.steps = steps_k;
                s.checks += 1;
                s.mass = tot[4];
                double res = tot[0] / d.u_ref;
                if (k.thermal) res = fmax(res, tot[2]);
                if (s.precise == 0 && res <= d.precise_from && tot[5] == 0 && isfinite(res)) {
                    // close enough to the steady state for round-off to freeze:
                    // switch to conserving, stochastically rounded increments
                    // (the mass is restored below) and restart the
                    // convergence bookkeeping for the remaining approach
                    s.precise = 2;
                    s.checks = 0;
                    s.res = s.res_prev = 0.0;
                    s.err_est = 1e30;
                    s.best_res = 1e300;
                    s.since_best = 0;
                    if (s.steps >= d.max_steps) s.state = kSlotMaxSteps;
                } else {
                // geometric extrapolation of the remaining change: with a
                // per-check contraction q = res / res_prev < 1, the distance
                // to the steady state is about res q / (1 - q); q from the
                // last two checks, the slower of the two contractions
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
                // the change stopped shrinking below tol / 4: the column has
                // reached the noise of the stochastic rounding (the check
                // interval makes the slowest mode's decay visible, so a flat
                // change is noise, not slow convergence)
                else if (s.since_best >= 8 && s.best_res <= 0.25 * d.tol) s.state = kSlotConverged;
                else if (s.since_best >= 50) s.state = kSlotStagnated;
                else if (s.steps >= d.max_steps) s.state = kSlotMaxSteps;
                }
            }
        }
        slot_barrier(CL);                      // the new state visible to the cluster
        if (__ldcg(&st->precise) == 2) {
            // the round-to-nearest phase let the column's mass drift by its
            // systematic round-off: restore the admission mass, spread over
            // the cells as rest equilibrium (d_a += dm w_a, no momentum)
            const float dm = (float)((d.mass0 - __ldcg(&st->mass)) / (double)Ny);
            float *f = const_cast<float *>(fin);
            for (int j = j0 + tid; j < j1; j += nth)
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    float &v = smem ? f[(j - j0) * Q + a] : f[(long long)a * Ny + j];
                    v = __fmaf_rn(dm, k.w[a], v);
                }
            slot_barrier(CL);                  // every CTA read precise == 2 and corrected
            if (rank == 0 && tid == 0) st->precise = 1;
            precise = 1;
        }
        return __ldcg(&st->state) == kSlotRunning;
    };
    // after sub-chunk kk of this launch: a check when the slot's chunk count
    // calls for one, else the counters (and the max_steps stop)
    auto after_chunk = [&](const float *fin, int kk) -> bool {
        const int ck = chunks0 + kk;
        const long long steps_k = steps0 + (long long)kk * chunk;
        if (ck % d.check_every == 0) return check(fin, ck, steps_k);
        if (rank == 0 && tid == 0) {
            st->chunks = ck;
            st->steps = steps_k;
            if (steps_k >= d.max_steps) st->state = kSlotMaxSteps;
        }
        return steps_k < d.max_steps;
    };

    float *g_cur = pool + d.f_off + (d.cur ? (long long)Q * Ny : 0);
    float *g_oth = pool + d.f_off + (d.cur ? 0 : (long long)Q * Ny);
    if (tid < 2) sw.acc[tid] = (float)k.accom[tid];
    int done = 0;
    if (smem) {
        // own rows into buffer 0, transposed to rows of Q populations
        for (int i = tid; i < Q * span; i += nth) {
            const int a = i / span, r = i - a * span;
            sm[r * Q + a] = __ldcg(g_cur + (long long)a * Ny + j0 + r);
        }
        const uint32_t base = (uint32_t)__cvta_generic_to_shared(sm);
        SmemState<Q> S{base, 0u, 0u, map_rank(base, rank), R, j0, 0};
        if (rank > 0) S.lo = map_rank(base, rank - 1);
        if (rank < CL - 1) S.hi = map_rank(base, rank + 1);
        slot_barrier(CL);                      // every CTA loaded before any neighbour reads
        while (done < d.sub) {
            const uint32_t s0 = (uint32_t)(steps0 + (long long)done * chunk);
            if (precise) run_steps<Q, true>(d, S, sw, chunk, CL, warp, lane, tid, nth, j0, j1, nb, nt, mb, me, s0);
            else run_steps<Q, false>(d, S, sw, chunk, CL, warp, lane, tid, nth, j0, j1, nb, nt, mb, me, s0);
            ++done;
            if (!after_chunk(sm + S.b * Q * R, done)) break;
        }
        // write the final state back to the pool buffer it came from
        const float *fin = sm + S.b * Q * R;
        for (int i = tid; i < Q * span; i += nth) {
            const int a = i / span, r = i - a * span;
            g_cur[(long long)a * Ny + j0 + r] = fin[r * Q + a];
        }
    } else {
        __syncthreads();
        GlobalState S{g_cur, g_oth, Ny, &sw.term[0][0][0]};
        while (done < d.sub) {
            const uint32_t s0 = (uint32_t)(steps0 + (long long)done * chunk);
            if (precise) run_steps<Q, true>(d, S, sw, chunk, CL, warp, lane, tid, nth, j0, j1, nb, nt, mb, me, s0);
            else run_steps<Q, false>(d, S, sw, chunk, CL, warp, lane, tid, nth, j0, j1, nb, nt, mb, me, s0);
            ++done;
            if (!after_chunk(S.src, done)) break;
        }
    }
    return done;
}

}  // namespace lbm
