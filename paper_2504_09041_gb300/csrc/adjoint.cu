// adjoint.cu -- launchers of the D2Q9 adjoint step and of its seed.
#include "adjoint_d2q9.cuh"
#include "kernels.h"

namespace lbm {

cudaError_t launch_adjoint_seed(const Geometry& geo, int face, double scale, void* mu, int arith,
                                cudaStream_t st)
{
    const int n_face = (face >> 1) == 0 ? geo.ny : geo.nx;
    const int nb = (n_face + 127) / 128;
    switch (arith) {
    case kAdjF64: adjoint_seed_d2q9_kernel<double><<<nb, 128, 0, st>>>((double*)mu, geo, face, scale); break;
    case kAdjF32: adjoint_seed_d2q9_kernel<float><<<nb, 128, 0, st>>>((float*)mu, geo, face, scale); break;
    case kAdjDF: adjoint_seed_d2q9_kernel<dfloat><<<nb, 128, 0, st>>>((dfloat*)mu, geo, face, scale); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class S, class RT>
static cudaError_t run_adjoint(const void* f_prev, const void* g_prev, const void* mu_in,
                               void* mu_out, const Geometry& geo, const HostCoeffs& hc,
                               int design_face, double* grad, cudaStream_t st)
{
    using T = typename S::T;
    using R = typename S::R;
    if (hc.adj_sync) {
        // thread blocks of the barrier-phased kernel: 64x4, 128x2, 32x4 or 64x2
        const int shapes[5][2] = {{0, 0}, {64, 4}, {128, 2}, {32, 4}, {64, 2}};
        const dim3 b(shapes[hc.adj_sync][0], shapes[hc.adj_sync][1], 1);
        const dim3 grid((geo.nx + b.x - 1) / b.x, (geo.ny + b.y - 1) / b.y, 1);
        adjoint_step_d2q9_kernel<S, RT, true><<<grid, b, 0, st>>>(
            (const T*)f_prev, (const T*)g_prev, (const RT*)mu_in, (RT*)mu_out, geo,
            make_coeffs<R, 9, 9>(hc), make_coeffs<TapeT<R, RT>, 9, 9>(hc), design_face, grad);
        return cudaGetLastError();
    }
    const dim3 b(64, 2, 1);
    const dim3 grid((geo.nx + b.x - 1) / b.x, (geo.ny + b.y - 1) / b.y, 1);
    adjoint_step_d2q9_kernel<S, RT><<<grid, b, 0, st>>>(
        (const T*)f_prev, (const T*)g_prev, (const RT*)mu_in, (RT*)mu_out, geo,
        make_coeffs<R, 9, 9>(hc), make_coeffs<TapeT<R, RT>, 9, 9>(hc), design_face, grad);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step_d2q9(int prec, int arith, const void* f_prev, const void* g_prev,
                                     const void* mu_in, void* mu_out, const Geometry& geo,
                                     const HostCoeffs& hc, int design_face, double* grad,
                                     cudaStream_t st)
{
#define LBM_ADJ(S)                                                                                  \
    switch (arith) {                                                                                \
    case kAdjF64: return run_adjoint<S, double>(f_prev, g_prev, mu_in, mu_out, geo, hc, design_face, grad, st); \
    case kAdjF32: return run_adjoint<S, float>(f_prev, g_prev, mu_in, mu_out, geo, hc, design_face, grad, st);  \
    case kAdjDF: return run_adjoint<S, dfloat>(f_prev, g_prev, mu_in, mu_out, geo, hc, design_face, grad, st); \
    }                                                                                               \
    return cudaErrorInvalidValue
    switch (prec) {
    case kF64: LBM_ADJ(StoreF64);
    case kF32: LBM_ADJ(StoreF32);
    case kF16S: LBM_ADJ(StoreF16S);
    }
#undef LBM_ADJ
    return cudaErrorInvalidValue;
}

}  // namespace lbm
