// Batched chunk kernel launch unit (one CTA per slot) and its per-slot
// initialisation and read-out kernels.
#include "batch_internal.h"
#include "k_aux.cuh"
#include "k_batch.cuh"

namespace lbm {

constexpr int kBatchThreads = 256;

// A slot descriptor is used only if its buffers lie inside the pool; a bad
// one is recorded in dbg[0..7] (code, slot, Q, Ny, f_off, prev_off, chunk,
// check interval) by the first CTA that meets it, and skipped.
__device__ __forceinline__ bool desc_ok(const SlotDesc &d, long long pool_elems, int slot,
                                        int code, int *dbg) {
    const bool q_ok = d.Q == 17 || d.Q == 25 || d.Q == 37;
    const long long need = 2LL * d.Q * d.Ny + 2LL * d.Ny;
    bool terms_ok = d.nterm >= 1 && d.nterm < 32 && d.nout >= 1 && d.nout <= kMaxOut;
    for (int w = 0; w < 2 && terms_ok; ++w) {
        for (int l = 0; l < d.nterm; ++l)
            terms_ok = terms_ok && d.term_a[w][l] >= 0 && d.term_a[w][l] < d.Q &&
                       d.term_row[w][l] >= 0 && d.term_row[w][l] < 3;
        for (int l = 0; l < d.nout; ++l)
            terms_ok = terms_ok && d.out_a[w][l] >= 0 && d.out_a[w][l] < d.Q;
    }
    bool mirror_ok = true;
    for (int a = 0; a < d.Q && q_ok; ++a)
        mirror_ok = mirror_ok && d.k.mirror[a] >= 0 && d.k.mirror[a] < d.Q;
    const bool cl_ok = batch_split_ok(d.Ny, d.cl);
    const bool ok = q_ok && terms_ok && mirror_ok && cl_ok && d.Ny >= 6 && d.Ny <= kMaxNy &&
                    d.sub >= 1 && d.sub <= kMaxSub &&
                    d.f_off >= 0 &&
                    d.f_off + need <= pool_elems && d.prev_off == d.f_off + 2LL * d.Q * d.Ny &&
                    (d.cur == 0 || d.cur == 1) && d.chunk_steps >= 1 && d.check_every >= 1;
    if (!ok && threadIdx.x == 0 && atomicCAS(dbg, 0, code) == 0) {
        dbg[1] = slot;
        dbg[2] = d.Q;
        dbg[3] = d.Ny;
        dbg[4] = (int)d.f_off;
        dbg[5] = (int)d.prev_off;
        dbg[6] = d.chunk_steps;
        dbg[7] = d.check_every;
    }
    return ok;
}

// Stage the slot descriptor in shared memory (broadcast reads afterwards).
__device__ __forceinline__ void load_desc(const SlotDesc *g, SlotDesc *s) {
    const int n = (int)(sizeof(SlotDesc) / sizeof(int));
    const int *src = (const int *)g;
    int *dst = (int *)s;
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// One chunk of slot slot0 + blockIdx.x / CL on a cluster of CL CTAs (CL = 1:
// a plain launch).  Every CTA of a cluster reads the same descriptor and
// status, so all of them take the same early exit or none does: no thread
// leaves while others of its cluster still meet barriers.
__global__ void __launch_bounds__(kBatchThreads, 2)
k_batch_chunk(SlotDesc *__restrict__ desc, SlotStatus *__restrict__ status,
              float *__restrict__ pool, double *__restrict__ part, int slot0, int CL,
              long long pool_elems, int *dbg) {
    __shared__ SlotDesc sd;
    __shared__ BatchWallShared sw;
    __shared__ int s_chunks, s_precise;
    __shared__ long long s_steps;
    extern __shared__ __align__(16) float batch_sm[];
    const int slot = slot0 + blockIdx.x / CL;
    const int rank = CL == 1 ? 0 : (int)cluster_rank();
    load_desc(desc + slot, &sd);
    if (threadIdx.x == 0) {
        s_chunks = status[slot].chunks;
        s_steps = status[slot].steps;
        s_precise = status[slot].precise;
    }
    __syncthreads();
    if (sd.Q == 0 || status[slot].state != kSlotRunning) return;
    if (!desc_ok(sd, pool_elems, slot, 1, dbg) || sd.cl != CL) return;
    double *pp = part + (long long)slot * (6 * kMaxResidualChunks);
    int done = 0;
    switch (sd.Q) {
    case 17: done = batch_slot<17>(sd, pool, status + slot, sw, rank, CL, s_chunks, s_steps, s_precise, pp, batch_sm); break;
    case 25: done = batch_slot<25>(sd, pool, status + slot, sw, rank, CL, s_chunks, s_steps, s_precise, pp, batch_sm); break;
    case 37: done = batch_slot<37>(sd, pool, status + slot, sw, rank, CL, s_chunks, s_steps, s_precise, pp, batch_sm); break;
    default: break;
    }
    // the global-memory path leaves the state in the other buffer after an odd
    // number of steps; the shared-memory path writes it back where it came from
    const bool smem = batch_uses_smem(sd.Ny, CL);
    if (!smem && rank == 0 && threadIdx.x == 0)
        desc[slot].cur = (int)((sd.cur + (long long)done * sd.chunk_steps) & 1);
}

// Initial state of newly admitted slots: the equilibrium f~* = rho0 g^eq(u, T)
// of Eq. (4) with u_x(y), T(y) from the descriptor (rest: u = 0, T = 1; the
// Sec. IV slip solution), stored as deviations from w_a; the previous-check
// fields are the initial u_x and T.
template <int Q>
__device__ void init_slot(const SlotDesc &d, float *pool, float rho0) {
    float *f = pool + d.f_off + (d.cur ? (long long)Q * d.Ny : 0);
    const bool thermal = d.k.thermal != 0;
    for (int j = threadIdx.x; j < d.Ny; j += blockDim.x) {
        const double y = (j + 0.5) / d.Ny;
        const float u = (float)(d.init_u0 + d.init_u1 * (y - 0.5));
        const float T = thermal ? (float)(d.init_T0 + d.init_T1 * y + d.init_T2 * y * (1.0 - y)) : 1.0f;
        float o[Q];
        equilibrium_all<Q, float, true>(rho0, rho0 - 1.0f, u, 0.0f, T, d.k, o);
#pragma unroll
        for (int a = 0; a < Q; ++a) f[(long long)a * d.Ny + j] = o[a];
        float *pu = pool + d.prev_off;
        pu[j] = u;
        pu[d.Ny + j] = T;
    }
}

__global__ void k_batch_init(SlotDesc *__restrict__ desc, float *__restrict__ pool,
                             const int *__restrict__ slots, float rho0, int nslots,
                             long long pool_elems, int *dbg) {
    __shared__ SlotDesc sd;
    const int slot = slots[blockIdx.x];
    if (slot < 0 || slot >= nslots) {
        if (threadIdx.x == 0 && atomicCAS(dbg, 0, 2) == 0) dbg[1] = slot;
        return;
    }
    load_desc(desc + slot, &sd);
    __syncthreads();
    if (!desc_ok(sd, pool_elems, slot, 3, dbg)) return;
    switch (sd.Q) {
    case 17: init_slot<17>(sd, pool, rho0); break;
    case 25: init_slot<25>(sd, pool, rho0); break;
    case 37: init_slot<37>(sd, pool, rho0); break;
    default: break;
    }
}

// Eq. (3) fields of finished slots into out[i][4][Ny] (FP64): rho, u_x, u_y, T.
template <int Q>
__device__ void macros_slot(const SlotDesc &d, const float *pool, double *out) {
    using L = Lat<Q>;
    const float *f = pool + d.f_off + (d.cur ? (long long)Q * d.Ny : 0);
    const double r = (double)d.k.r;
    for (int j = threadIdx.x; j < d.Ny; j += blockDim.x) {
        // stored deviations d = f - w
        double s0 = 0, sx = 0, sy = 0, se = (double)d.k.e2w;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double fa = (double)f[(long long)a * d.Ny + j];
            s0 += fa;
            sx += L::ex(a) * fa;
            sy += L::ey(a) * fa;
            se += L::e2(a) * fa;
        }
        const double rh = 1.0 + s0;
        const double u = r * sx / rh, v = r * sy / rh;
        out[j] = rh;
        out[d.Ny + j] = u;
        out[2 * d.Ny + j] = v;
        out[3 * d.Ny + j] = ((double)d.k.r2 * se - rh * (u * u + v * v)) / (2.0 * rh);
    }
}

__global__ void k_batch_macros(const SlotDesc *__restrict__ desc, const float *__restrict__ pool,
                               const int *__restrict__ slots, const long long *__restrict__ out_off,
                               double *__restrict__ out, int nslots, long long pool_elems,
                               long long out_elems, int *dbg) {
    __shared__ SlotDesc sd;
    const int slot = slots[blockIdx.x];
    if (slot < 0 || slot >= nslots) {
        if (threadIdx.x == 0 && atomicCAS(dbg, 0, 4) == 0) dbg[1] = slot;
        return;
    }
    load_desc(desc + slot, &sd);
    __syncthreads();
    if (!desc_ok(sd, pool_elems, slot, 5, dbg)) return;
    if (out_off[blockIdx.x] < 0 || out_off[blockIdx.x] + 4LL * sd.Ny > out_elems) {
        if (threadIdx.x == 0 && atomicCAS(dbg, 0, 6) == 0) {
            dbg[1] = slot;
            dbg[3] = sd.Ny;
            dbg[4] = (int)out_off[blockIdx.x];
        }
        return;
    }
    double *o = out + out_off[blockIdx.x];
    switch (sd.Q) {
    case 17: macros_slot<17>(sd, pool, o); break;
    case 25: macros_slot<25>(sd, pool, o); break;
    case 37: macros_slot<37>(sd, pool, o); break;
    default: break;
    }
}

// Load the batch kernels' module now (not lazily during a stream capture).
int preload_batch_kernels() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncSetAttribute(k_batch_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_chunk, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_batch_chunk);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_batch_init);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_batch_macros);
    return (int)e;
}

int batch_max_cluster() {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, (const void *)k_batch_chunk, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();                    // not an error of the caller's
        return 8;
    }
    return n >= 1 ? 16 : 8;
}

int launch_batch_chunk(cudaStream_t st, SlotDesc *desc, SlotStatus *status, float *pool,
                       double *part, int slot0, int nlanes, int CL, long long pool_elems,
                       int *dbg) {
    if (nlanes <= 0) return 0;
    if (CL == 1) {
        k_batch_chunk<<<nlanes, kBatchThreads, kSmemBytes, st>>>(desc, status, pool, part, slot0,
                                                                 1, pool_elems, dbg);
        return (int)cudaGetLastError();
    }
    if (CL != 2 && CL != 4 && CL != 8 && CL != 16) return (int)cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nlanes * CL));
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, k_batch_chunk, desc, status, pool, part, slot0, CL,
                                   pool_elems, dbg);
}

int launch_batch_init(cudaStream_t st, SlotDesc *desc, float *pool, const int *slots, int n,
                      float rho0, int nslots, long long pool_elems, int *dbg) {
    if (n <= 0) return 0;
    k_batch_init<<<n, kBatchThreads, 0, st>>>(desc, pool, slots, rho0, nslots, pool_elems, dbg);
    return (int)cudaGetLastError();
}

int launch_batch_macros(cudaStream_t st, const SlotDesc *desc, const float *pool,
                        const int *slots, const long long *out_off, double *out, int n,
                        int nslots, long long pool_elems, long long out_elems, int *dbg) {
    if (n <= 0) return 0;
    k_batch_macros<<<n, kBatchThreads, 0, st>>>(desc, pool, slots, out_off, out, nslots,
                                                pool_elems, out_elems, dbg);
    return (int)cudaGetLastError();
}

}  // namespace lbm
