// step2d.cu -- instantiations of the fused D2Q9 flow + D2Q9 energy step.
#include "kernels.h"
#include "step_d2q9.cuh"

namespace lbm {

template <class S>
static cudaError_t run(const void* fin, const void* gin, void* fout, void* gout, const Geometry& geo,
                       const HostCoeffs& hc, unsigned* status, dim3 block, cudaStream_t st)
{
    using T = typename S::T;
    using R = typename S::R;
    const dim3 b = block_shape(geo.nx, block);
    const dim3 grid((geo.nx + b.x - 1) / b.x, (geo.ny + b.y - 1) / b.y, 1);
    const auto c = make_coeffs<R, 9, 9>(hc);
    if (step_index32(geo, 9, hc))
        step_d2q9_kernel<S, unsigned><<<grid, b, 0, st>>>((const T*)fin, (const T*)gin, (T*)fout,
                                                          (T*)gout, geo, c, status);
    else
        step_d2q9_kernel<S, size_t><<<grid, b, 0, st>>>((const T*)fin, (const T*)gin, (T*)fout,
                                                        (T*)gout, geo, c, status);
    return cudaGetLastError();
}

cudaError_t launch_step_d2q9(int prec, const void* fin, const void* gin, void* fout, void* gout,
                             const Geometry& geo, const HostCoeffs& hc, unsigned* status,
                             dim3 block, cudaStream_t st)
{
    switch (prec) {
    case kF64: return run<StoreF64>(fin, gin, fout, gout, geo, hc, status, block, st);
    case kF32: return run<StoreF32>(fin, gin, fout, gout, geo, hc, status, block, st);
    case kF16S: return run<StoreF16S>(fin, gin, fout, gout, geo, hc, status, block, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
