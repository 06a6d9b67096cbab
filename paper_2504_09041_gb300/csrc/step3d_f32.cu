// step3d_f32.cu -- the fused D3Q27 flow + D3Q15 energy step with StoreF32 storage (one
// translation unit per storage type so that the three heavy instantiations compile in parallel).
#include <algorithm>

#include "kernels.h"
#include "step_d3q27_tma.cuh"

namespace lbm {

// kU: the collision instance for the rates (rate_class: 0 general, 1 unit-rate energy collision,
// 2 unit-rate energy collision and flow relaxation).
template <int kU>
static cudaError_t launch_plain_f32(const void* fin, const void* gin, void* fout, void* gout,
                                  const Geometry& geo, const HostCoeffs& hc, unsigned* status,
                                  dim3 block, cudaStream_t st)
{
    using S = StoreF32;
    using T = typename S::T;
    using R = typename S::R;
    const dim3 b = block_shape(geo.nx, block, 3);
    const auto c = make_coeffs<R, 27, 15>(hc);
    const int rows = rows3d_for(hc, false);
    if (step_index32(geo, 27, hc) && rows == 2) {
        dim3 g = grid_shape(geo, b);
        g.y = (g.y + 1) / 2;
        step_d3q27_kernel<S, unsigned, 2, kU><<<g, b, 0, st>>>(
            (const T*)fin, (const T*)gin, (T*)fout, (T*)gout, geo, c, status);
    } else if (step_index32(geo, 27, hc) && rows == 4) {
        dim3 g = grid_shape(geo, b);
        g.y = (g.y + 3) / 4;
        step_d3q27_kernel<S, unsigned, 4, kU><<<g, b, 0, st>>>(
            (const T*)fin, (const T*)gin, (T*)fout, (T*)gout, geo, c, status);
    } else if (step_index32(geo, 27, hc))
        step_d3q27_kernel<S, unsigned, 1, kU><<<grid_shape(geo, b), b, 0, st>>>(
            (const T*)fin, (const T*)gin, (T*)fout, (T*)gout, geo, c, status);
    else
        step_d3q27_kernel<S, size_t, 1, kU><<<grid_shape(geo, b), b, 0, st>>>(
            (const T*)fin, (const T*)gin, (T*)fout, (T*)gout, geo, c, status);
    return cudaGetLastError();
}

cudaError_t launch_step_d3q27_f32(const void* fin, const void* gin, void* fout, void* gout,
                                  const Geometry& geo, const HostCoeffs& hc, unsigned* status,
                                  dim3 block, cudaStream_t st)
{
    switch (rate_class(hc)) {
    case 2: return launch_plain_f32<2>(fin, gin, fout, gout, geo, hc, status, block, st);
    case 1: return launch_plain_f32<1>(fin, gin, fout, gout, geo, hc, status, block, st);
    }
    return launch_plain_f32<0>(fin, gin, fout, gout, geo, hc, status, block, st);
}

template <int TY, int kU>
static cudaError_t launch_tma_f32(const TmaMaps& tm, const void* fin, const void* gin, void* fout,
                                  void* gout, const Geometry& geo, const HostCoeffs& hc,
                                  unsigned* status, cudaStream_t st)
{
    using S = StoreF32;
    using T = typename S::T;
    using R = typename S::R;
    using L = TmaLayout<T, TY>;
    const auto c = make_coeffs<R, 27, 15>(hc);
    const int tiles_x = (geo.nx + kTmaTX - 1) / kTmaTX, tiles_y = (geo.ny + TY - 1) / TY;
    const int n_tiles = tiles_x * tiles_y * geo.nz;
    const dim3 block(kTmaTX * TY + 32, 1, 1);   // TY rows of consumers and one producer warp
    auto kern = step_index32(geo, 27, hc) ? step_d3q27_tma_kernel<S, unsigned, TY, kU>
                                          : step_d3q27_tma_kernel<S, size_t, TY, kU>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTmaTX * TY + 32, L::kSmemBytes)) != cudaSuccess)
        return e;
    const int grid = std::max(1, std::min(n_tiles, sms * std::max(1, per_sm)));
    kern<<<grid, block, L::kSmemBytes, st>>>(tm.f, tm.g, (const T*)fin, (const T*)gin, (T*)fout, (T*)gout,
                                            geo, c, status, tiles_x, tiles_y, n_tiles);
    return cudaGetLastError();
}

template <int kU>
static cudaError_t launch_tma_rows_f32(const TmaMaps& tm, const void* fin, const void* gin, void* fout,
                                       void* gout, const Geometry& geo, const HostCoeffs& hc,
                                       unsigned* status, cudaStream_t st)
{
    switch (tm.ty) {
    case 1: return launch_tma_f32<1, kU>(tm, fin, gin, fout, gout, geo, hc, status, st);
    case 2: return launch_tma_f32<2, kU>(tm, fin, gin, fout, gout, geo, hc, status, st);
    case 4: return launch_tma_f32<4, kU>(tm, fin, gin, fout, gout, geo, hc, status, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_d3q27_tma_f32(const TmaMaps& tm, const void* fin, const void* gin, void* fout,
                                      void* gout, const Geometry& geo, const HostCoeffs& hc,
                                      unsigned* status, cudaStream_t st)
{
    switch (rate_class(hc)) {
    case 2: return launch_tma_rows_f32<2>(tm, fin, gin, fout, gout, geo, hc, status, st);
    case 1: return launch_tma_rows_f32<1>(tm, fin, gin, fout, gout, geo, hc, status, st);
    }
    return launch_tma_rows_f32<0>(tm, fin, gin, fout, gout, geo, hc, status, st);
}

}  // namespace lbm
