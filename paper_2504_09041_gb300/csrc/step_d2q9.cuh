// step_d2q9.cuh -- fused pull-stream + FP central-moment collision of the coupled D2Q9 flow
// (Appendix A) and D2Q9 energy (Appendix B) lattices, one node per thread.
//
// The raw -> central map of Steps 1-2 is done as two sweeps of 3-link lines (x, then y), which
// equals P then F on the tensor-product D2Q9 set; Steps 4-5 are the inverse sweeps.
//
// Deviation form: the kernel carries delta_a = f_a - w_a and gamma_a = g_a - w_a T_o.  Because
// the sweeps are linear, the central moments of f are those of the rest populations w at the
// velocity u, K_ab = W_a(ux) W_b(uy) with W_0 = 1, W_1 = -u, W_2 = 1/3 + u^2, plus the central
// moments D_ab of delta.  The relaxation is rewritten for the deviations D_ab -> T_ab
// (kappa~_ab = K_ab + T_ab) with the O(1) parts of K cancelled analytically, so every quantity
// in the collision is small and keeps the register type's full relative precision.
#pragma once

#include "lattices.cuh"
#include "lbm_common.cuh"

namespace lbm {

template <class R>
using Coeffs2D = Coeffs<R, 9, 9>;

// Streaming (Eqs. LBMsteps-stream, LBMsteps-streamg) with half-way bounce-back for f, and
// bounce-back (adiabatic) or anti-bounce-back (fixed T) for g at the walls (Sec. 6.1), in
// deviations: the anti-bounce-back g_a = -g~_abar + 2 w_a T_w becomes
// gamma_a = -gamma~_abar + 2 w_a (T_w - T_o).
template <class S, class Idx = size_t>
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
        const Idx off = out ? (Idx)o * geo.n + i : (Idx)a * geo.n + s;
        f[a] = S::load_dev(fin, off, R(w9(a)));
        const R gv = S::load_dev(gin, off, R(w9(a)) * T_ref);
        g[a] = dir ? R(2.0 * w9(a)) * (tw - T_ref) - gv : gv;
    });
}

// The same pull at a node whose eight neighbours all lie inside the box: no wall and no
// periodic wrap touches any link, so every population comes straight from its upwind node.
template <class S, class Idx = size_t>
__device__ __forceinline__ void pull_d2q9_interior(const typename S::T* __restrict__ fin,
                                                   const typename S::T* __restrict__ gin,
                                                   const Geometry& geo, int i, typename S::R T_ref,
                                                   typename S::R f[9], typename S::R g[9])
{
    using R = typename S::R;
    static_for<9>([&](auto A) {
        constexpr int a = decltype(A)::value;
        const Idx off = (Idx)a * geo.n + (i - (e9(a, 0) + e9(a, 1) * geo.nx));
        f[a] = S::load_dev(fin, off, R(w9(a)));
        g[a] = S::load_dev(gin, off, R(w9(a)) * T_ref);
    });
}

// Flow collision (App. A Step 3; second-order sources vanish; sigma_12 carries the factor 2 of
// Eq. forcing:2D) on the deviations: D[b][a] = kappa_ab - K_ab on entry, kappa~_ab - K_ab on exit.
template <class R>
__device__ __forceinline__ void relax_f_d2q9(R D[3][3], R drho, R irho, R ux, R uy, R Fx, R Fy,
                                             const Coeffs2D<R>& c)
{
    const R third = R(1.0 / 3.0);
    const R A = third + ux * ux, B = third + uy * uy;     // K_20, K_02
    const R uxuy = ux * uy;                                // K_11
    const R D00 = D[0][0], D10 = D[0][1], D20 = D[0][2];
    const R D01 = D[1][0], D11 = D[1][1], D21 = D[1][2];
    const R D02 = D[2][0], D12 = D[2][1], D22 = D[2][2];
    const R Fxr = Fx * irho, Fyr = Fy * irho;
    // sources with the full pre-collision moments kappa = K + D
    const R k11 = uxuy + D11, k20 = A + D20, k02 = B + D02;
    const R k21 = D21 - A * uy, k12 = D12 - ux * B;
    const R s21 = R(2) * Fxr * k11 + Fyr * k20;
    const R s12 = Fxr * k02 + R(2) * Fyr * k11;
    const R s22 = R(2) * (Fxr * k12 + Fyr * k21);

    const R T00 = D00 + c.om_f[0] * (drho - D00);
    const R T10 = D10 - c.om_f[1] * (D10 - ux) + c.hf[1] * Fx;
    const R T01 = D01 - c.om_f[2] * (D01 - uy) + c.hf[2] * Fy;
    const R D2s = D20 + D02, D2d = D20 - D02;
    const R u2s = ux * ux + uy * uy, u2d = ux * ux - uy * uy;
    const R T2s = D2s + c.om_f[3] * (R(2.0 / 3.0) * drho - u2s - D2s);
    const R T2d = D2d - c.om_f[4] * (D2d + u2d);
    const R T11 = D11 - c.om_f[5] * (D11 + uxuy);
    const R T21 = D21 - c.om_f[6] * (D21 - A * uy) + c.hf[6] * s21;
    const R T12 = D12 - c.om_f[7] * (D12 - ux * B) + c.hf[7] * s12;
    const R T20 = R(0.5) * (T2s + T2d);
    const R T02 = R(0.5) * (T2s - T2d);
    // kappa^Mv_22 - K_22 with t20 = A + T20, t02 = B + T02, t11 = uxuy + T11
    const R t11 = uxuy + T11;
    const R M22 = (A * T02 + B * T20 + T20 * T02 + R(2) * t11 * t11 - A * B * drho) * irho;
    const R T22 = D22 + c.om_f[8] * (M22 - D22) + c.hf[8] * s22;

    D[0][0] = T00; D[0][1] = T10; D[0][2] = T20;
    D[1][0] = T01; D[1][1] = T11; D[1][2] = T21;
    D[2][0] = T02; D[2][1] = T12; D[2][2] = T22;
}

// Energy collision in central-moment space on full values (App. B Step 3); n[b][a] holds eta_ab
// on entry and eta~_ab on exit.  The attractors of orders 3-4 come from the post-collision lower
// moments: option A (Eq. MvT2D, c.gopt = 0) or the renormalized option B (Eq. MvT2DoptionB).
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
    R Mv21, Mv12, Mv22;
    if (c.gopt == 0) {
        Mv21 = R(2.0 / 3.0 * cs2) * t01;
        Mv12 = R(2.0 / 3.0 * cs2) * t10;
        Mv22 = R(0.5 * cs2) * (t20 + t02);
    } else {
        const R iT = R(1) / T;
        const R c23 = R(2.0 / 3.0) * iT;
        Mv21 = c23 * (t20 * t01 + R(2) * t11 * t10);
        Mv12 = c23 * (t02 * t10 + R(2) * t11 * t01);
        Mv22 = iT * (t20 * t02 + R(2) * t11 * t11);
    }
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

// One time step at one node: pull, macroscopic fields (App. A Step 7, App. B Step 7, Sec. 6.1
// Boussinesq force), collide f and g, store.
template <class S, class Idx>
__device__ __forceinline__ void node_step_d2q9(const typename S::T* __restrict__ fin,
                                               const typename S::T* __restrict__ gin,
                                               typename S::T* __restrict__ fout,
                                               typename S::T* __restrict__ gout, const Geometry& geo,
                                               const Coeffs2D<typename S::R>& c, unsigned* status,
                                               int x, int y)
{
    using R = typename S::R;
    const int i = x + geo.nx * y;
    R f[9], g[9];
    // Which pull: decided per warp where possible, so that a warp holding an x-wall node of an
    // interior row runs one x-only pull instead of both the interior and the general pull.
    const bool y_in = y > 0 && y < geo.ny - 1;
    const bool in = y_in && x > 0 && x < geo.nx - 1;
    const unsigned lanes = __activemask();
    if (__all_sync(lanes, in)) {
        pull_d2q9_interior<S, Idx>(fin, gin, geo, i, c.T_ref, f, g);
    } else if (__all_sync(lanes, y_in)) {
        const NodeWalls<R> w = node_walls_x<R>(geo, x, y, 0);
        pull_d2q9<S, Idx>(fin, gin, geo, w, i, c.T_ref, f, g);
    } else if (in) {
        pull_d2q9_interior<S, Idx>(fin, gin, geo, i, c.T_ref, f, g);
    } else {
        const NodeWalls<R> w = node_walls<R>(geo, x, y, 0, 2);
        pull_d2q9<S, Idx>(fin, gin, geo, w, i, c.T_ref, f, g);
    }

    // rho = 1 + sum delta, rho u = sum delta e + F/2, T = T_o + sum gamma (sum w = 1, sum w e = 0)
    const R dT = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const R drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const R jx = (f[1] + f[5] + f[8]) - (f[3] + f[6] + f[7]);
    const R jy = (f[2] + f[5] + f[6]) - (f[4] + f[7] + f[8]);
    const R Fb = c.gbeta * dT;
    const R Fx = c.gaxis == 0 ? Fb : R(0);
    const R Fy = c.gaxis == 1 ? Fb : R(0);
    const R rho = R(1) + drho;
    const R T = c.T_ref + dT;
    const R irho = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * irho;
    const R uy = (jy + R(0.5) * Fy) * irho;
    check_node(status, rho, T);

    R p[3][3];
    to_central_d2q9(f, p, ux, uy);
    relax_f_d2q9(p, drho, irho, ux, uy, Fx, Fy, c);
    from_central_d2q9(p, f, ux, uy);

    // energy populations on full values: g = w T_o + gamma
    static_for<9>([&](auto A) {
        constexpr int a = decltype(A)::value;
        g[a] += R(w9(a)) * c.T_ref;
    });
    to_central_d2q9(g, p, ux, uy);
    relax_g_d2q9(p, T, c);
    from_central_d2q9(p, g, ux, uy);

    if constexpr (std::is_same<S, StoreF16S>::value) {
        if (c.fp16_sr) {
            R dg[9];
            static_for<9>([&](auto A) {
                constexpr int a = decltype(A)::value;
                dg[a] = g[a] - R(w9(a)) * c.T_ref;
            });
            store_node_f16s_sr<9, 9, Idx>(fout, gout, (Idx)geo.n, i, f, dg);
            return;
        }
    }
    static_for<9>([&](auto A) {
        constexpr int a = decltype(A)::value;
        S::store_dev(fout, (Idx)a * geo.n + i, f[a], R(w9(a)));
        S::store_dev(gout, (Idx)a * geo.n + i, g[a] - R(w9(a)) * c.T_ref, R(w9(a)) * c.T_ref);
    });
}

template <class S, class Idx>
__global__ void __launch_bounds__(256)
    step_d2q9_kernel(const typename S::T* __restrict__ fin, const typename S::T* __restrict__ gin,
                     typename S::T* __restrict__ fout, typename S::T* __restrict__ gout, Geometry geo,
                     Coeffs2D<typename S::R> c, unsigned* status)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= geo.nx || y >= geo.ny) return;
    node_step_d2q9<S, Idx>(fin, gin, fout, gout, geo, c, status, x, y);
}

}  // namespace lbm
