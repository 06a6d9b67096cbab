// step_d2q9.cuh -- fused pull-stream + FP central-moment collision of the coupled D2Q9 flow
// (Appendix A) and D2Q9 energy (Appendix B) lattices, one node per thread.
//
// The raw -> central map of Steps 1-2 is done as two sweeps of 3-link lines (x, then y), which
// equals P then F on the tensor-product D2Q9 set; Steps 4-5 are the inverse sweeps.
#pragma once

#include "lattices.cuh"
#include "lbm_common.cuh"

namespace lbm {

template <class R>
using Coeffs2D = Coeffs<R, 9, 9>;

// Streaming (Eqs. LBMsteps-stream, LBMsteps-streamg) with half-way bounce-back for f, and
// bounce-back (adiabatic) or anti-bounce-back (fixed T) for g at the walls (Sec. 5.1).
template <class S>
__device__ __forceinline__ void pull_d2q9(const typename S::T* __restrict__ fin,
                                          const typename S::T* __restrict__ gin, const Geometry& geo,
                                          const NodeWalls<typename S::R>& w, int i, typename S::R T_ref,
                                          typename S::R f[9], typename S::R g[9])
{
    using R = typename S::R;
    static_for<9>([&](auto A) {
        constexpr int a = decltype(A)::value;
        constexpr int o = opp9(a);
        bool out, dir;
        R tw;
        const int s = link_source<e9(a, 0), e9(a, 1), 0>(geo, w, i, &out, &dir, &tw);
        const size_t off = out ? (size_t)o * geo.n + i : (size_t)a * geo.n + s;
        f[a] = S::load(fin, off, R(w9(a)));
        const R gv = S::load(gin, off, R(w9(a)) * T_ref);
        g[a] = dir ? R(2.0 * w9(a)) * tw - gv : gv;
    });
}

// Flow collision in central-moment space (App. A Step 3, readings R5 and R8 of the oracle's
// notes: second-order sources vanish, sigma_12 carries the factor 2 of Eq. forcing:2D).
// k[b][a] holds kappa_ab on entry and kappa~_ab on exit.
template <class R>
__device__ __forceinline__ void relax_f_d2q9(R k[3][3], R rho, R irho, R Fx, R Fy, const Coeffs2D<R>& c)
{
    const R k00 = k[0][0], k10 = k[0][1], k20 = k[0][2];
    const R k01 = k[1][0], k11 = k[1][1], k21 = k[1][2];
    const R k02 = k[2][0], k12 = k[2][1], k22 = k[2][2];
    const R Fxr = Fx * irho, Fyr = Fy * irho;
    const R s21 = R(2) * Fxr * k11 + Fyr * k20;
    const R s12 = Fxr * k02 + R(2) * Fyr * k11;
    const R s22 = R(2) * (Fxr * k12 + Fyr * k21);

    const R t00 = k00 + c.om_f[0] * (rho - k00);
    const R t10 = k10 - c.om_f[1] * k10 + c.hf[1] * Fx;
    const R t01 = k01 - c.om_f[2] * k01 + c.hf[2] * Fy;
    const R k2s = k20 + k02, k2d = k20 - k02;
    const R t2s = k2s + c.om_f[3] * (R(2.0 / 3.0) * rho - k2s);
    const R t2d = k2d - c.om_f[4] * k2d;
    const R t11 = k11 - c.om_f[5] * k11;
    const R t21 = k21 - c.om_f[6] * k21 + c.hf[6] * s21;
    const R t12 = k12 - c.om_f[7] * k12 + c.hf[7] * s12;
    const R t20 = R(0.5) * (t2s + t2d);
    const R t02 = R(0.5) * (t2s - t2d);
    const R Mv22 = (t20 * t02 + R(2) * t11 * t11) * irho;
    const R t22 = k22 + c.om_f[8] * (Mv22 - k22) + c.hf[8] * s22;

    k[0][0] = t00; k[0][1] = t10; k[0][2] = t20;
    k[1][0] = t01; k[1][1] = t11; k[1][2] = t21;
    k[2][0] = t02; k[2][1] = t12; k[2][2] = t22;
}

// Energy collision in central-moment space (App. B Step 3, option-A attractors Eq. MvT2D).
template <class R>
__device__ __forceinline__ void relax_g_d2q9(R n[3][3], R T, const Coeffs2D<R>& c)
{
    const R n00 = n[0][0], n10 = n[0][1], n20 = n[0][2];
    const R n01 = n[1][0], n11 = n[1][1], n21 = n[1][2];
    const R n02 = n[2][0], n12 = n[2][1], n22 = n[2][2];
    constexpr double cs2 = 1.0 / 3.0;

    const R t00 = n00 + c.om_g[0] * (T - n00);
    const R t10 = n10 - c.om_g[1] * n10;
    const R t01 = n01 - c.om_g[2] * n01;
    const R n2s = n20 + n02, n2d = n20 - n02;
    const R t2s = n2s + c.om_g[3] * (R(2 * cs2) * T - n2s);
    const R t2d = n2d - c.om_g[4] * n2d;
    const R t11 = n11 - c.om_g[5] * n11;
    const R t20 = R(0.5) * (t2s + t2d);
    const R t02 = R(0.5) * (t2s - t2d);
    const R Mv21 = R(2.0 / 3.0 * cs2) * t01;
    const R Mv12 = R(2.0 / 3.0 * cs2) * t10;
    const R Mv22 = R(0.5 * cs2) * (t20 + t02);
    const R t21 = n21 + c.om_g[6] * (Mv21 - n21);
    const R t12 = n12 + c.om_g[7] * (Mv12 - n12);
    const R t22 = n22 + c.om_g[8] * (Mv22 - n22);

    n[0][0] = t00; n[0][1] = t10; n[0][2] = t20;
    n[1][0] = t01; n[1][1] = t11; n[1][2] = t21;
    n[2][0] = t02; n[2][1] = t12; n[2][2] = t22;
}

// Populations (paper order) <-> p[ey+1][ex+1], then the x and y line sweeps.
template <class R>
__device__ __forceinline__ void to_central_d2q9(const R f[9], R p[3][3], R ux, R uy)
{
    static_for<9>([&](auto A) {
        constexpr int a = decltype(A)::value;
        p[e9(a, 1) + 1][e9(a, 0) + 1] = f[a];
    });
#pragma unroll
    for (int j = 0; j < 3; ++j) central_line(p[j][0], p[j][1], p[j][2], ux);
#pragma unroll
    for (int a = 0; a < 3; ++a) central_line(p[0][a], p[1][a], p[2][a], uy);
}

template <class R>
__device__ __forceinline__ void from_central_d2q9(R p[3][3], R f[9], R ux, R uy)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) uncentral_line(p[0][a], p[1][a], p[2][a], uy);
#pragma unroll
    for (int j = 0; j < 3; ++j) uncentral_line(p[j][0], p[j][1], p[j][2], ux);
    static_for<9>([&](auto A) {
        constexpr int a = decltype(A)::value;
        f[a] = p[e9(a, 1) + 1][e9(a, 0) + 1];
    });
}

// One time step at one node: pull, macroscopic fields (App. A Step 7, App. B Step 7, Sec. 5.1
// Boussinesq force), collide f and g, store.
template <class S>
__device__ __forceinline__ void node_step_d2q9(const typename S::T* __restrict__ fin,
                                               const typename S::T* __restrict__ gin,
                                               typename S::T* __restrict__ fout,
                                               typename S::T* __restrict__ gout, const Geometry& geo,
                                               const Coeffs2D<typename S::R>& c, unsigned* status,
                                               int x, int y)
{
    using R = typename S::R;
    const int i = x + geo.nx * y;
    const NodeWalls<R> w = node_walls<R>(geo, x, y, 0, 2);
    R f[9], g[9];
    pull_d2q9<S>(fin, gin, geo, w, i, c.T_ref, f, g);

    const R T = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const R rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const R jx = (f[1] + f[5] + f[8]) - (f[3] + f[6] + f[7]);
    const R jy = (f[2] + f[5] + f[6]) - (f[4] + f[7] + f[8]);
    const R Fb = c.gbeta * (T - c.T_ref);
    const R Fx = c.gaxis == 0 ? Fb : R(0);
    const R Fy = c.gaxis == 1 ? Fb : R(0);
    const R irho = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * irho;
    const R uy = (jy + R(0.5) * Fy) * irho;
    check_node(status, rho, T);

    R p[3][3];
    to_central_d2q9(f, p, ux, uy);
    relax_f_d2q9(p, rho, irho, Fx, Fy, c);
    from_central_d2q9(p, f, ux, uy);

    to_central_d2q9(g, p, ux, uy);
    relax_g_d2q9(p, T, c);
    from_central_d2q9(p, g, ux, uy);

    static_for<9>([&](auto A) {
        constexpr int a = decltype(A)::value;
        S::store(fout, (size_t)a * geo.n + i, f[a], R(w9(a)));
        S::store(gout, (size_t)a * geo.n + i, g[a], R(w9(a)) * c.T_ref);
    });
}

template <class S>
__global__ void __launch_bounds__(256)
    step_d2q9_kernel(const typename S::T* __restrict__ fin, const typename S::T* __restrict__ gin,
                     typename S::T* __restrict__ fout, typename S::T* __restrict__ gout, Geometry geo,
                     Coeffs2D<typename S::R> c, unsigned* status)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= geo.nx || y >= geo.ny) return;
    node_step_d2q9<S>(fin, gin, fout, gout, geo, c, status, x, y);
}

}  // namespace lbm
