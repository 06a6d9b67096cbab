// tma.cu -- tensor-map encoding for the TMA-staged 3D step, through the driver entry point that
// the CUDA runtime exposes (no link against the driver library).
#include <cstdio>
#include <mutex>
#include <string>

#include "kernels.h"

namespace lbm {

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                 CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                 CUtensorMapFloatOOBfill);

EncodeTiled encoder(std::string* err)
{
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    static std::string why;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                               cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            why = "cuTensorMapEncodeTiled is not available from the driver";
        else
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    if (!fn && err) *err = why;
    return fn;
}

}  // namespace

bool make_tma_map(CUtensorMap* out, void* base, int elem_bytes, int nx, int ny, int nz, int planes,
                  int ty, std::string* err)
{
    if ((long long)nx * elem_bytes % 16 != 0) {
        if (err) *err = "the TMA-staged step needs nx * element size to be a multiple of 16 bytes";
        return false;
    }
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) {
        if (err) *err = "population buffer is not 16-byte aligned";
        return false;
    }
    EncodeTiled enc = encoder(err);
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)planes};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * elem_bytes, (cuuint64_t)nx * ny * elem_bytes,
                                   (cuuint64_t)nx * ny * nz * elem_bytes};
    // 64 nodes of tile plus 16 bytes of nodes on each side (step_d3q27_tma.cuh)
    const cuuint32_t box[4] = {(cuuint32_t)(64 + 32 / elem_bytes), (cuuint32_t)ty, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const CUresult r = enc(out, dt, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (err) {
            char buf[96];
            snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
            *err = buf;
        }
        return false;
    }
    return true;
}

}  // namespace lbm
