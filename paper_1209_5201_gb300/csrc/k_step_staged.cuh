// TMA-staged, warp-specialised, persistent tile kernel of a full time step
// (Eq. (5) pull-stream + Eq. (3)-(4) collision + Eq. (12) diffuse wall).
//
// Tile: TX columns x TY rows of fluid cells.  For velocity a the tile pulls
// the source window shifted by (-e_ax, -e_ay): rows j0 - e_ay .. +TY and
// columns x0 - 4 .. x0 + TX + 4 of velocity a, i.e. the tile plus the x-halo
// rounded to 16 bytes.  Grids stored as one x-tile only (their row segments
// hold every column; see KConsts).  One elected producer thread stages the Q
// windows of a tile with 3-D TMA boxes (x, a, y) into a ring of STAGES shared-memory
// buffers; rows outside [0, Ny) arrive zero-filled and are replaced by the
// diffuse-wall fill.  Consumer warps read their cell's Q values from shared
// memory (conflict-free, consecutive lanes on consecutive columns), release
// the buffer, collide and write the Q post-collision values with coalesced
// stores.  BF16DEV also stages the FP32 density plane with its +-3-row halo.
//
// Every mbarrier wait is bounded (KConsts::wait_ns, 2 s unless the host sets
// another limit): on expiry the thread records an error code in *err and the
// CTA stops taking tiles; the producer then waits for its copies in flight
// before exiting, with a fixed 2 s limit of its own.
#pragma once

#include <cuda.h>

#include "lbm_device.cuh"

namespace lbm {

constexpr int kStagedErrTimeout = 1;
constexpr unsigned long long kDrainWaitNs = kDefaultWaitNs;   // copies in flight at exit

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: false when limit_ns ran out; a zero limit gives up at once,
// whether or not the phase has completed (the failure path, on demand)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns) {
    if (limit_ns == 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cta.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}

template <int Q, int PREC, int TX, int TY, int STAGES, int CPT>
struct StagedCfg {
    using S = typename Store<PREC>::S;
    static constexpr int kW = TX + 2 * kPadL;                   // staged row width
    static constexpr int kBoxBytes = kW * TY * (int)sizeof(S);  // one plane window
    static constexpr int kPlaneStride = (kBoxBytes + 127) / 128 * 128;
    static constexpr bool kDev = Store<PREC>::dev;
    static constexpr int kRhoRows = TY + 6;
    static constexpr int kRhoBytes = kDev ? kW * kRhoRows * 4 : 0;
    static constexpr int kRhoStride = (kRhoBytes + 127) / 128 * 128;
    static constexpr int kStageBytes = Q * kPlaneStride + kRhoStride;
    static constexpr int kTxBytes = Q * kBoxBytes + kRhoBytes;  // bytes TMA delivers
    static constexpr int kConsumers = TX * TY / CPT;
    static constexpr int kConsumerWarps = kConsumers / 32;
    static constexpr int kThreads = kConsumers + 32;
    // 128 bytes of slack for aligning the dynamic base, 1 KB of barriers,
    // the stage ring, and the two walls' incoming-mass sums
    static constexpr int kSmem = 128 + 1024 + STAGES * kStageBytes + 2 * (TX + 6) * 8;
    static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
    static_assert(kConsumers % 32 == 0, "consumer threads must fill warps");
    static_assert(TX % 32 == 0, "tile width must be a multiple of 32 columns");
    static_assert(kW * (int)sizeof(S) % 16 == 0, "TMA rows must be 16-byte multiples");
    static_assert(kStageBytes % 128 == 0, "stage alignment");
};

template <int Q, int PREC, int TX, int TY, int STAGES, int CPT>
__global__ void __launch_bounds__(StagedCfg<Q, PREC, TX, TY, STAGES, CPT>::kThreads, 1)
k_step_staged(const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_r,
              const typename Store<PREC>::S *__restrict__ fin,
              typename Store<PREC>::S *__restrict__ fout, const float *__restrict__ rin,
              float *__restrict__ rout, int *__restrict__ err,
              const __grid_constant__ KConsts<typename Store<PREC>::C> k) {
    using Cfg = StagedCfg<Q, PREC, TX, TY, STAGES, CPT>;
    using L = Lat<Q>;
    using S = typename Store<PREC>::S;
    using C = typename Store<PREC>::C;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 1 KB header: barriers; then the stage ring; then the wall sums
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t *full = (uint64_t *)base;
    uint64_t *empty = full + STAGES;
    uint64_t *wbar = empty + STAGES;        // consumers' barrier around the wall sums
    int *stop = (int *)(wbar + 1);
    unsigned char *ring = base + 1024;
    double *s_min = (double *)(ring + STAGES * Cfg::kStageBytes);   // [2][TX + 6]

    const int ntx = (k.Nx + TX - 1) / TX;
    const int nty = (k.Ny + TY - 1) / TY;
    const int ntiles = ntx * nty;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp == Cfg::kConsumerWarps;
    // BF16: step count of the stochastic rounding (block 0 advances it)
    uint32_t seed = 0;
    if constexpr (Store<PREC>::sr) seed = step_count(fin, k, blockIdx.x == 0 && threadIdx.x == 0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], Cfg::kConsumerWarps);
        }
        mbar_init(wbar, Cfg::kConsumers);
        *stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (producer) {
        if (lane == 0) {
            int it = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (it >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, k.wait_ns)) {
                    atomicOr(err, kStagedErrTimeout);
                    *(volatile int *)stop = 1;
                    break;
                }
                if (*(volatile int *)stop) break;
                const int x0 = (t % ntx) * TX, j0 = (t / ntx) * TY;
                unsigned char *st = ring + s * Cfg::kStageBytes;
                mbar_arrive_expect_tx(&full[s], Cfg::kTxBytes);
#pragma unroll
                for (int a = 0; a < Q; ++a)
                    tma_load_3d(st + a * Cfg::kPlaneStride, &tm_f, &full[s], x0, a, j0 - L::ey(a));
                if constexpr (Cfg::kDev)
                    tma_load_2d(st + Q * Cfg::kPlaneStride, &tm_r, &full[s], x0, j0 - 3);
            }
            // drain: every issued stage must have landed before the CTA exits
            // (its own fixed limit, whatever the limit of the other waits)
            const int issued = it;
            for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; ++i)
                if (!mbar_wait(&full[i % STAGES], (uint32_t)(i / STAGES) & 1u, kDrainWaitNs))
                    atomicOr(err, kStagedErrTimeout);
        }
        return;
    }

    // ---- consumers --------------------------------------------------------------
    const int tid = threadIdx.x;
    uint32_t wphase = 0;
    auto wall_sync = [&]() -> bool {
        mbar_arrive(wbar);
        const bool ok = mbar_wait(wbar, wphase, k.wait_ns);
        wphase ^= 1u;
        return ok;
    };
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        const int x0 = (t % ntx) * TX, j0 = (t / ntx) * TY;
        const bool wb = j0 < L::N, wt = j0 + TY > k.Ny - L::N;
        if (wb || wt) {
            // Eq. (12) numerator for ghost columns x0 - 3 .. x0 + TX + 2, FP64;
            // the first barrier keeps the previous wall tile's readers safe
            if (!wall_sync()) {
                atomicOr(err, kStagedErrTimeout);
                *(volatile int *)stop = 1;
                break;
            }
            for (int w = 0; w < 2; ++w) {
                if (!(w == 0 ? wb : wt)) continue;
                for (int c = tid; c < TX + 6; c += Cfg::kConsumers) {
                    const int xw = wrap(x0 - 3 + c, k.Nx);
                    double m = 0.0;
#pragma unroll
                    for (int b = 0; b < Q; ++b) {
                        const int eyb = L::ey(b);
                        if (w == 0 ? !(eyb < 0) : !(eyb > 0)) continue;
                        const int xs = wrap(xw - L::ex(b), k.Nx);
                        const int depth = eyb < 0 ? -eyb : eyb;
                        for (int kk = 0; kk < depth; ++kk) {
                            const int row = w == 0 ? kk : k.Ny - 1 - kk;
                            double v = (double)to_c(
                                fin[col_index(k, row, xs) + (long long)b * k.pitch]);
                            if constexpr (Cfg::kDev)
                                v += (double)k.w[b] * (double)rin[rho_index(k, row, xs)];
                            if constexpr (Store<PREC>::shifted) v += (double)k.w[b];
                            m += v;
                        }
                    }
                    s_min[w * (TX + 6) + c] = m;
                }
            }
            if (!wall_sync()) {
                atomicOr(err, kStagedErrTimeout);
                *(volatile int *)stop = 1;
                break;
            }
        }
        if (!mbar_wait(&full[s], ph, k.wait_ns)) {
            atomicOr(err, kStagedErrTimeout);
            *(volatile int *)stop = 1;
            break;
        }
        const unsigned char *st = ring + s * Cfg::kStageBytes;
        const float *srho = (const float *)(st + Q * Cfg::kPlaneStride);

        C fv[CPT][Q];
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int cell = tid + q * Cfg::kConsumers;
            const int i = cell % TX, kr = cell / TX;
            const int j = j0 + kr;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const int sj = j - L::ey(a);
                if ((wb || wt) && (sj < 0 || sj >= k.Ny)) {
                    const int wall = sj < 0 ? 0 : 1;
                    const C spec = (k.accom[wall] != 1.0 && x0 + i < k.Nx && j < k.Ny)
                                       ? specular_source<PREC>(fin, rin, k, a, L::ex(a), x0 + i, j)
                                       : C(0);
                    fv[q][a] = wall_mix<PREC>(s_min[wall * (TX + 6) + i + 3 - L::ex(a)],
                                              k.wcoef[wall][a], k.w[a], k.accom[wall], spec);
                } else {
                    const S *pl = (const S *)(st + a * Cfg::kPlaneStride);
                    C v = to_c(pl[kr * Cfg::kW + i + kPadL - L::ex(a)]);
                    if constexpr (Cfg::kDev)
                        v = dev_to_f(v, k.w[a], srho[(kr + 3 - L::ey(a)) * Cfg::kW + i + kPadL - L::ex(a)]);
                    fv[q][a] = v;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);

#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int cell = tid + q * Cfg::kConsumers;
            const int i = cell % TX, kr = cell / TX;
            const int x = x0 + i, j = j0 + kr;
            if (x >= k.Nx || j >= k.Ny) continue;
            Collision<Q, C, Store<PREC>::shifted> col;
            col.setup(fv[q], k);
            C o[Q];
            o[0] = col.rest(fv[q][0]);
            PairLoop<1, Q>::run([&](auto ic) {
                constexpr int A = decltype(ic)::value;
                col.template pair<A>(fv[q][A], fv[q][A + 1], o[A], o[A + 1]);
            });
            const uint32_t hcell = Store<PREC>::sr ? sr_cell(seed, (uint32_t)j * (uint32_t)k.Nx + (uint32_t)x) : 0u;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                C v = o[a];
                if constexpr (Cfg::kDev) v = f_to_dev(v, k.w[a], col.rho);
                store_pop<S>(fout, k, a, j, x, store_rounded<S>(v, sr_bits(hcell, a)));
            }
            if constexpr (Cfg::kDev) store_rho(rout, k, j, x, (float)col.rho);
        }
        if (*(volatile int *)stop) break;
    }
}

}  // namespace lbm
