// Batched chunk kernel launch unit (one CTA per slot) and its per-slot
// initialisation and read-out kernels.
#include "batch_internal.h"
#include "k_batch.cuh"

namespace lbm {

constexpr int kBatchThreads = 256;

// Stage the slot descriptor in shared memory (broadcast reads afterwards).
__device__ __forceinline__ void load_desc(const SlotDesc *g, SlotDesc *s) {
    const int n = (int)(sizeof(SlotDesc) / sizeof(int));
    const int *src = (const int *)g;
    int *dst = (int *)s;
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

__global__ void __launch_bounds__(kBatchThreads, 2)
k_batch_chunk(SlotDesc *__restrict__ desc, SlotStatus *__restrict__ status,
              float *__restrict__ pool, int chunk) {
    __shared__ SlotDesc sd;
    __shared__ double s_min[2];
    __shared__ int s_term[128];
    const int slot = blockIdx.x;
    load_desc(desc + slot, &sd);
    __syncthreads();
    if (sd.Q == 0 || status[slot].state != kSlotRunning) return;
    switch (sd.Q) {
    case 17: batch_slot<17>(sd, pool, status + slot, chunk, s_min, s_term); break;
    case 25: batch_slot<25>(sd, pool, status + slot, chunk, s_min, s_term); break;
    case 37: batch_slot<37>(sd, pool, status + slot, chunk, s_min, s_term); break;
    default: break;
    }
    if (threadIdx.x == 0) desc[slot].cur = (sd.cur + chunk) & 1;
}

// Rest equilibrium f~* = rho0 w_a of newly admitted slots; previous-check
// fields u_x = 0, T = 1.
template <int Q>
__device__ void init_slot(const SlotDesc &d, float *pool, float rho0) {
    float *f = pool + d.f_off + (d.cur ? (long long)Q * d.Ny : 0);
    for (int j = threadIdx.x; j < d.Ny; j += blockDim.x) {
#pragma unroll
        for (int a = 0; a < Q; ++a) f[(long long)a * d.Ny + j] = rho0 * d.k.w[a];
        float *pu = pool + d.prev_off;
        pu[j] = 0.0f;
        pu[d.Ny + j] = 1.0f;
    }
}

__global__ void k_batch_init(SlotDesc *__restrict__ desc, float *__restrict__ pool,
                             const int *__restrict__ slots, float rho0) {
    __shared__ SlotDesc sd;
    load_desc(desc + slots[blockIdx.x], &sd);
    __syncthreads();
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
        double fv[Q], s0 = 0, sx = 0, sy = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            fv[a] = f[(long long)a * d.Ny + j];
            s0 += fv[a];
            sx += L::ex(a) * fv[a];
            sy += L::ey(a) * fv[a];
        }
        const double u = r * sx / s0, v = r * sy / s0;
        double e = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double cx = r * L::ex(a) - u, cy = r * L::ey(a) - v;
            e += fv[a] * (cx * cx + cy * cy);
        }
        out[j] = s0;
        out[d.Ny + j] = u;
        out[2 * d.Ny + j] = v;
        out[3 * d.Ny + j] = e / (2.0 * s0);
    }
}

__global__ void k_batch_macros(const SlotDesc *__restrict__ desc, const float *__restrict__ pool,
                               const int *__restrict__ slots, const long long *__restrict__ out_off,
                               double *__restrict__ out) {
    __shared__ SlotDesc sd;
    load_desc(desc + slots[blockIdx.x], &sd);
    __syncthreads();
    double *o = out + out_off[blockIdx.x];
    switch (sd.Q) {
    case 17: macros_slot<17>(sd, pool, o); break;
    case 25: macros_slot<25>(sd, pool, o); break;
    case 37: macros_slot<37>(sd, pool, o); break;
    default: break;
    }
}

int launch_batch_chunk(cudaStream_t st, SlotDesc *desc, SlotStatus *status, float *pool,
                       int nslots, int chunk) {
    if (nslots <= 0) return 0;
    k_batch_chunk<<<nslots, kBatchThreads, 0, st>>>(desc, status, pool, chunk);
    return (int)cudaGetLastError();
}

int launch_batch_init(cudaStream_t st, SlotDesc *desc, float *pool, const int *slots, int n,
                      float rho0) {
    if (n <= 0) return 0;
    k_batch_init<<<n, kBatchThreads, 0, st>>>(desc, pool, slots, rho0);
    return (int)cudaGetLastError();
}

int launch_batch_macros(cudaStream_t st, const SlotDesc *desc, const float *pool,
                        const int *slots, const long long *out_off, double *out, int n) {
    if (n <= 0) return 0;
    k_batch_macros<<<n, kBatchThreads, 0, st>>>(desc, pool, slots, out_off, out);
    return (int)cudaGetLastError();
}

}  // namespace lbm
