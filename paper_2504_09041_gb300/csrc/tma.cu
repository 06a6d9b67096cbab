// tma.cu -- tensor-map encoding for the TMA-staged 3D step, through the driver entry point that
// the CUDA runtime exposes (no link against the driver library).
#include <cstdio>
#include <mutex>
#include <string>

#include "kernels.h"
#include "step_d3q27_tma.cuh"

namespace lbm {

// One thread waits, bounded, on an mbarrier that nothing arrives on.
__global__ void probe_wait_kernel(long long limit_cycles, unsigned* result)
{
    __shared__ __align__(8) unsigned long long bar;
    const unsigned b = smem_addr(&bar);
    mbar_init(b, 1);
    fence_mbar_init();
    const bool done = mbar_wait_bounded(b, 0, limit_cycles);
    *result = done ? 0u : 2u;
}

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

extern "C" int lbm_probe_bounded_wait(double seconds, int* timed_out)
{
    if (!timed_out || !(seconds > 0.0 && seconds <= 10.0)) return LBM_EINVAL;
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    unsigned* r = nullptr;
    if (cudaMalloc(&r, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ENOMEM;
    }
    const long long limit = (long long)(seconds * 1e3 * (double)khz);
    lbm::probe_wait_kernel<<<1, 1>>>(limit, r);
    unsigned out = 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&out, r, sizeof out, cudaMemcpyDeviceToHost);
    cudaFree(r);
    if (e != cudaSuccess) return LBM_ECUDA;
    *timed_out = out == 2u ? 1 : 0;
    return out == 2u ? LBM_ETIMEOUT : LBM_OK;
}
