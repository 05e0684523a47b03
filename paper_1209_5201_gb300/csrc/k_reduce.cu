// Precision-independent kernels: FP64 reductions for the steady-state
// residual and mass drift, and the density plane of the BF16 deviation format.
#include "k_aux.cuh"
#include "launchers.h"

namespace lbm {

int reduction_blocks(long long n) {
    long long b = (n + kAuxThreads - 1) / kAuxThreads;
    if (b > 1024) b = 1024;
    return (int)(b < 1 ? 1 : b);
}

__global__ void k_accumulate(double *acc, const double *in, long long n, int first) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x)
        acc[c] = first ? in[c] : acc[c] + in[c];
}

__global__ void k_rho_plane_from_f64(float *rplane, const double *acc,
                                     const __grid_constant__ KConsts<float> k) {
    const long long n = (long long)k.Nx * k.Ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / k.Nx), x = (int)(c % k.Nx);
        store_rho(rplane, k, j, x, (float)acc[c]);
    }
}

// Sum nv-vectors of per-block partials in block order (one block).
__global__ void k_final_sum(const double *partials, int nblocks, int nv, double *out) {
    for (int i = 0; i < nv; ++i) {
        double v[1] = {0.0};
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v[0] += partials[(long long)b * nv + i];
        block_sum<1>(v, out + i);
        __syncthreads();
    }
}

// Residual partials over FP64 field planes: sum (ux - uxp)^2, sum ux^2,
// sum (T - Tp)^2, sum (T - Tref)^2, count of non-finite values; then the
// current fields become the previous ones.
__global__ void k_residual_partials(const double *ux, const double *T, double *uxp, double *Tp,
                                    long long n, double Tref, double *partials) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const double u = ux[c], t = T[c];
        const double du = u - uxp[c], dt = t - Tp[c], tr = t - Tref;
        acc[0] += du * du;
        acc[1] += u * u;
        acc[2] += dt * dt;
        acc[3] += tr * tr;
        if (!isfinite(u) || !isfinite(t)) acc[4] += 1.0;
        uxp[c] = u;
        Tp[c] = t;
    }
    block_sum<5>(acc, partials + (long long)blockIdx.x * 5);
}

int launch_accumulate(cudaStream_t st, double *acc, const double *in, long long n, int first) {
    k_accumulate<<<reduction_blocks(n), kAuxThreads, 0, st>>>(acc, in, n, first);
    return (int)cudaGetLastError();
}

int launch_rho_plane(cudaStream_t st, float *rplane, const double *acc, const KConsts<float> &k) {
    k_rho_plane_from_f64<<<reduction_blocks((long long)k.Nx * k.Ny), kAuxThreads, 0, st>>>(
        rplane, acc, k);
    return (int)cudaGetLastError();
}

int launch_final_sum(cudaStream_t st, const double *partials, int nblocks, int nv, double *out) {
    k_final_sum<<<1, kAuxThreads, 0, st>>>(partials, nblocks, nv, out);
    return (int)cudaGetLastError();
}

int launch_residual_partials(cudaStream_t st, const double *ux, const double *T, double *uxp,
                             double *Tp, long long n, double Tref, double *partials,
                             int nblocks) {
    k_residual_partials<<<nblocks, kAuxThreads, 0, st>>>(ux, T, uxp, Tp, n, Tref, partials);
    return (int)cudaGetLastError();
}

}  // namespace lbm
