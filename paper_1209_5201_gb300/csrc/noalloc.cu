// Steady-state residual reduction that allocates no memory.
//
// Same FP64 reduction as the solver's residual check (block partials in a
// fixed order, then one block sums them), but its scratch is the file-scope
// device array below instead of memory the library or the caller allocates.
// The array is created when the library is loaded and lives on every GPU
// that loads it until the process exits.
#include <mutex>

#include "k_aux.cuh"
#include "launchers.h"

namespace lbm {

constexpr int kNoAllocBlocks = 1024;        // block partials the array can hold
constexpr int kNoAllocVals = 5;             // sums per block
constexpr long long kNoAllocMaxCells = 2147483647LL;

// 1024 x 5 block partials + 8 totals = 41,024 bytes per device
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocBlocks * kNoAllocVals + 8];

namespace {

std::mutex g_mu;
double *g_addr[128] = {};                   // device address of the array, per device

// res = ||u - u'|| / ||u|| (thermal: max with ||T - T'|| / ||T - T_ref||);
// NaN when any field value was not finite
__global__ void k_residual_finish(const double *tot, int thermal, double *res) {
    double r = sqrt(tot[0]) / fmax(sqrt(tot[1]), 1e-30);
    if (thermal) r = fmax(r, sqrt(tot[2]) / fmax(sqrt(tot[3]), 1e-30));
    res[0] = tot[4] > 0 ? nan("") : r;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_residual_noalloc(const double *ux, const double *T, double *ux_prev,
                                    double *T_prev, int64_t n, double T_ref, int32_t thermal,
                                    double *res, void *stream) {
    if (!ux || !T || !ux_prev || !T_prev || !res) {
        set_error("lbm_residual_noalloc: NULL pointer");
        return LBM_EINVAL;
    }
    if (n < 1 || n > kNoAllocMaxCells) {
        set_error("lbm_residual_noalloc: n must be in [1, 2^31 - 1]");
        return LBM_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        set_error("lbm_residual_noalloc: no usable current device");
        return LBM_ECUDA;
    }
    double *scratch;
    {
        // first call on a device: look up the array's device address (with that
        // device current); later calls reuse it
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_error(std::string("lbm_residual_noalloc: cudaGetSymbolAddress: ") +
                          cudaGetErrorString(e));
                return LBM_ECUDA;
            }
            g_addr[dev] = (double *)p;
        }
        scratch = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = reduction_blocks(n);           // capped at kNoAllocBlocks
    if (nb > kNoAllocBlocks) {
        set_error("lbm_residual_noalloc: too many block partials for the scratch array");
        return LBM_EINVAL;
    }
    double *partials = scratch;
    double *tot = scratch + kNoAllocBlocks * kNoAllocVals;
    // every partial and total is overwritten by this call, nothing needs clearing
    if ((e = (cudaError_t)launch_residual_partials(st, ux, T, ux_prev, T_prev, n, T_ref, partials, nb)) ||
        (e = (cudaError_t)launch_final_sum(st, partials, nb, kNoAllocVals, tot))) {
        set_error(std::string("lbm_residual_noalloc: ") + cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    k_residual_finish<<<1, 1, 0, st>>>(tot, thermal, res);
    if ((e = cudaGetLastError())) {
        set_error(std::string("lbm_residual_noalloc: ") + cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    return LBM_OK;
}
