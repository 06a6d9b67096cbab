// step3d_f64.cu -- the fused D3Q27 flow + D3Q15 energy step with StoreF64 storage (one
// translation unit per storage type so that the three heavy instantiations compile in parallel).
#include "kernels.h"
#include "step_d3q27.cuh"

namespace lbm {

// kU: the collision instance for the rates (rate_class: 0 general, 1 unit-rate energy collision,
// 2 unit-rate energy collision and flow relaxation).
template <int kU>
static cudaError_t launch_plain_f64(const void* fin, const void* gin, void* fout, void* gout,
                                    const Geometry& geo, const HostCoeffs& hc, unsigned* status,
                                    dim3 block, cudaStream_t st)
{
    using S = StoreF64;
    using T = typename S::T;
    using R = typename S::R;
    const dim3 b = block_shape(geo.nx, block, 3);
    const auto c = make_coeffs<R, 27, 15>(hc);
    if (step_index32(geo, 27, hc))
        step_d3q27_kernel<S, unsigned, 1, kU><<<grid_shape(geo, b), b, 0, st>>>(
            (const T*)fin, (const T*)gin, (T*)fout, (T*)gout, geo, c, status);
    else
        step_d3q27_kernel<S, size_t, 1, kU><<<grid_shape(geo, b), b, 0, st>>>(
            (const T*)fin, (const T*)gin, (T*)fout, (T*)gout, geo, c, status);
    return cudaGetLastError();
}

cudaError_t launch_step_d3q27_f64(const void* fin, const void* gin, void* fout, void* gout,
                                  const Geometry& geo, const HostCoeffs& hc, unsigned* status,
                                  dim3 block, cudaStream_t st)
{
    switch (rate_class(hc)) {
    case 2: return launch_plain_f64<2>(fin, gin, fout, gout, geo, hc, status, block, st);
    case 1: return launch_plain_f64<1>(fin, gin, fout, gout, geo, hc, status, block, st);
    }
    return launch_plain_f64<0>(fin, gin, fout, gout, geo, hc, status, block, st);
}

}  // namespace lbm
