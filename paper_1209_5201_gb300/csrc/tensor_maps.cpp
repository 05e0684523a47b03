// Tensor maps of the TMA-staged step kernel.  cuTensorMapEncodeTiled is a
// driver entry point; it is fetched through the runtime so that the library
// needs no link against libcuda.
#include <cudaTypedefs.h>

#include <string>

#include "lbm_internal.h"

namespace lbm {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}
}  // namespace

int encode_tensor_maps(SolverImpl &s, int TX, int TY) {
    const long long key = (long long)TX * 4096 + TY;
    if (s.tm_key == key) return 0;
    auto enc = encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled entry point unavailable");
        return LBM_ECUDA;
    }
    const CUtensorMapDataType dt = s.p.precision == LBM_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : s.p.precision == LBM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t es = (cuuint64_t)s.elem;
    const cuuint32_t W = (cuuint32_t)(TX + 2 * kPadL);
    for (int b = 0; b < 2; ++b) {
        // one x-tile: element (a, j, p) at (j Q + a) pitch + p; dims (p, a, j)
        cuuint64_t dims[3] = {(cuuint64_t)s.pitch, (cuuint64_t)s.L.Q, (cuuint64_t)s.p.Ny};
        cuuint64_t strides[2] = {(cuuint64_t)s.pitch * es, (cuuint64_t)s.pitch * s.L.Q * es};
        cuuint32_t box[3] = {W, 1, (cuuint32_t)TY};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = enc(&s.tm_f[b], dt, 3, s.f[b], dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled (state) failed: " + std::to_string((int)r));
            return LBM_ECUDA;
        }
        if (s.rho[b]) {
            cuuint64_t rd[2] = {(cuuint64_t)s.pitch, (cuuint64_t)s.p.Ny};
            cuuint64_t rs[1] = {(cuuint64_t)s.pitch * 4};
            cuuint32_t rb[2] = {W, (cuuint32_t)(TY + 6)};
            cuuint32_t re[2] = {1, 1};
            r = enc(&s.tm_r[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, s.rho[b], rd, rs, rb, re,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                set_error("cuTensorMapEncodeTiled (density) failed: " + std::to_string((int)r));
                return LBM_ECUDA;
            }
        }
    }
    s.tm_key = key;
    return 0;
}

}  // namespace lbm
