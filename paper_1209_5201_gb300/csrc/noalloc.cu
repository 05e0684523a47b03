// Steady-state residual reduction that allocates no memory.
//
// Same FP64 reduction as the solver's residual check (block partials in a
// fixed order, then one block sums them), but its scratch is the file-scope
// device array below instead of memory the library or the caller allocates.
// The array is created when the library is loaded and lives on every GPU
// that loads it until the process exits.
#include <cudaTypedefs.h>

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
// The array's device address is a property of the CUDA context it was loaded
// into: a context the caller created and made current, or the primary context
// re-created after cudaDeviceReset, holds its own copy at another address.  So
// the address is cached with the unique ID of the context it was looked up in
// (cuCtxGetId: unique for the life of the process), and looked up again when
// the current context's ID differs.
struct CachedAddr {
    unsigned long long ctx_id;
    double *addr;
};
CachedAddr g_addr[128] = {};                // per device: last context and address

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// driver entry points, fetched through the runtime (no link against libcuda)
template <class F>
F driver_fn(const char *name, int version) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return (F)p;
}

// unique ID of the calling thread's current context; an error (with a
// message unless quiet) if none is current
int current_context_id(unsigned long long &id, bool quiet = false) {
    static CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent", 4000);
    static CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId", 12000);
    if (!get_current || !get_id) {
        set_error("lbm_residual_noalloc: driver entry points cuCtxGetCurrent / cuCtxGetId unavailable");
        return LBM_ECUDA;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || get_id(ctx, &id) != CUDA_SUCCESS) {
        if (!quiet) set_error("lbm_residual_noalloc: no current CUDA context");
        return LBM_ECUDA;
    }
    return LBM_OK;
}

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
        // first call in a context: look up the array's device address there
        // (the look-up also binds the runtime's context to this thread when
        // none is current yet); later calls in the same context reuse it
        std::lock_guard<std::mutex> lk(g_mu);
        unsigned long long ctx_id = 0;
        const bool bound = current_context_id(ctx_id, true) == LBM_OK;
        if (!bound || !g_addr[dev].addr || g_addr[dev].ctx_id != ctx_id) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_error(std::string("lbm_residual_noalloc: cudaGetSymbolAddress: ") +
                          cudaGetErrorString(e));
                return LBM_ECUDA;
            }
            if (!bound)
                if (int rc = current_context_id(ctx_id)) return rc;
            g_addr[dev] = CachedAddr{ctx_id, (double *)p};
        }
        scratch = g_addr[dev].addr;
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
