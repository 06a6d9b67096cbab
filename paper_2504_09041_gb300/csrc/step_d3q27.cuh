// step_d3q27.cuh -- fused pull-stream + FP central-moment collision of the coupled D3Q27 flow
// (Sec. 5.1-5.2) and D3Q15 energy (Appendix C) lattices, one node per thread.
//
// D3Q27: the 27 central moments kappa_abc are produced by three sweeps of 3-link lines (x, y, z),
// which on the tensor-product lattice equals P then F; the inverse sweeps map back.
// D3Q15: raw moments come from the six axis links in pairs and from an 8-point Walsh-Hadamard
// transform of the corner links (the structure of App. C Step 1); the central shift and its exact
// inverse are applied axis by axis (Steps 2 and 4, including the aliased moment 220).
//
// Deviation form: the kernel carries delta_a = f_a - w_a and gamma_b = g_b - w_b T_o.  The central
// moments of f are those of the rest populations at the velocity u, K_abc = W_a(ux) W_b(uy)
// W_c(uz) with W_0 = 1, W_1 = -u, W_2 = 1/3 + u^2, plus the central moments D_abc of delta; the
// flow relaxation is written for the deviations with the O(1) parts of K (the moments even in
// every direction) cancelled analytically, so the FP32 arithmetic resolves the small departures
// from rest.
#pragma once

#include "lattices.cuh"
#include "lbm_common.cuh"

#ifndef LBM_MAXREG3D
#define LBM_MAXREG3D Launch3D<S, kRates>::kMaxRegs
#endif

namespace lbm {

template <class R>
using Coeffs3D = Coeffs<R, 27, 15>;

// D3Q15 link b for D3Q27 link a, or -1.
__host__ __device__ constexpr int g15_of_27(int a)
{
    return a < 7 ? a : (a >= 19 ? a - 12 : -1);
}

template <class S, class Idx = size_t>
__device__ __forceinline__ void pull_d3q27_d3q15(const typename S::T* __restrict__ fin,
                                                 const typename S::T* __restrict__ gin,
                                                 const Geometry& geo,
                                                 const NodeWalls<typename S::R>& w, int i,
                                                 typename S::R T_ref, typename S::R f[27],
                                                 typename S::R g[15])
{
    using R = typename S::R;
    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        constexpr int o = opp27(a);
        bool out, dir;
        R tw;
        const int s = link_source<e27(a, 0), e27(a, 1), e27(a, 2)>(geo, w, i, &out, &dir, &tw);
        const Idx off = out ? (Idx)o * geo.n + i : (Idx)a * geo.n + s;
        f[a] = S::load_dev(fin, off, R(w27(a)));
        constexpr int b = g15_of_27(a);
        if constexpr (b >= 0) {
            constexpr int ob = opp15(b);
            const Idx og = out ? (Idx)ob * geo.n + i : (Idx)b * geo.n + s;
            const R gv = S::load_dev(gin, og, R(w15(b)) * T_ref);
            g[b] = dir ? R(2.0 * w15(b)) * (tw - T_ref) - gv : gv;
        }
    });
}

// The same pull at a node whose 26 neighbours all lie inside the box (no wall, no wrap).
template <class S, class Idx = size_t>
__device__ __forceinline__ void pull_d3q27_d3q15_interior(const typename S::T* __restrict__ fin,
                                                          const typename S::T* __restrict__ gin,
                                                          const Geometry& geo, int i,
                                                          typename S::R T_ref, typename S::R f[27],
                                                          typename S::R g[15])
{
    using R = typename S::R;
    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        const int s = i - (e27(a, 0) + e27(a, 1) * geo.nx + e27(a, 2) * geo.nxy);
        f[a] = S::load_dev(fin, (Idx)a * geo.n + s, R(w27(a)));
        constexpr int b = g15_of_27(a);
        if constexpr (b >= 0) g[b] = S::load_dev(gin, (Idx)b * geo.n + s, R(w15(b)) * T_ref);
    });
}

// Flow collision (reading R6 of the oracle notes) on the deviations: D[c][b][a] = kappa_abc - K_abc
// on entry, kappa~_abc - K_abc on exit.  Rate slots follow the moment order of Sec. 5.2; slot 7
// relaxes the trace (bulk), slots 8 and 9 the deviators kappa_200 - kappa_020, kappa_200 - kappa_002.
// Sources (Eq. forcing:3D) use the full pre-collision moments kappa = K + D.
// kUnit: the rates are those of lbm_create (every rate 1 except the shear ones, slots 4-6, 8, 9;
// unit_flow_rates), which the host has checked.  A moment relaxed at rate 1 lands on its attractor
// plus half its source, so its pre-collision value drops out of its own update (order 6 drops out
// entirely).
template <bool kUnit = false, class R>
__device__ __forceinline__ void relax_f_d3q27(R D[3][3][3], R drho, R irho, R ux, R uy, R uz, R Fx,
                                              R Fy, R Fz, const Coeffs3D<R>& c)
{
    const R hu = R(0.5);   // 1 - omega / 2 at omega = 1
#define DD(a, b, cc) D[cc][b][a]
    const R* om = c.om_f;
    const R* h = c.hf;
    const R third = R(1.0 / 3.0);
    const R Fxr = Fx * irho, Fyr = Fy * irho, Fzr = Fz * irho;
    // rest moments at u: W_2 per axis, products of W_1
    const R A = third + ux * ux, B = third + uy * uy, C = third + uz * uz;
    const R xy = ux * uy, xz = ux * uz, yz = uy * uz;

    // pre-collision deviations
    const R d000 = DD(0, 0, 0), d100 = DD(1, 0, 0), d010 = DD(0, 1, 0), d001 = DD(0, 0, 1);
    const R d110 = DD(1, 1, 0), d101 = DD(1, 0, 1), d011 = DD(0, 1, 1);
    const R d200 = DD(2, 0, 0), d020 = DD(0, 2, 0), d002 = DD(0, 0, 2);
    const R d120 = DD(1, 2, 0), d102 = DD(1, 0, 2), d210 = DD(2, 1, 0), d012 = DD(0, 1, 2);
    const R d201 = DD(2, 0, 1), d021 = DD(0, 2, 1), d111 = DD(1, 1, 1);
    const R d220 = DD(2, 2, 0), d202 = DD(2, 0, 2), d022 = DD(0, 2, 2);
    const R d211 = DD(2, 1, 1), d121 = DD(1, 2, 1), d112 = DD(1, 1, 2);
    const R d122 = DD(1, 2, 2), d212 = DD(2, 1, 2), d221 = DD(2, 2, 1), d222 = DD(2, 2, 2);

    // full pre-collision moments needed by the sources
    const R k110 = xy + d110, k101 = xz + d101, k011 = yz + d011;
    const R k200 = A + d200, k020 = B + d020, k002 = C + d002;
    const R k120 = d120 - ux * B, k102 = d102 - ux * C, k210 = d210 - A * uy;
    const R k012 = d012 - uy * C, k201 = d201 - A * uz, k021 = d021 - B * uz;
    const R k111 = d111 - xy * uz;
    const R k220 = A * B + d220;
    const R k211 = A * yz + d211, k121 = B * xz + d121, k112 = C * xy + d112;
    const R k022 = B * C + d022, k202 = A * C + d202;
    const R k122 = d122 - ux * B * C, k212 = d212 - A * uy * C, k221 = d221 - A * B * uz;

    // orders 0 and 1 (K_000 = 1, K_100 = -ux, ...)
    const R t000 = kUnit ? drho : d000 + om[0] * (drho - d000);
    const R t100 = kUnit ? ux + hu * Fx : d100 - om[1] * (d100 - ux) + h[1] * Fx;
    const R t010 = kUnit ? uy + hu * Fy : d010 - om[2] * (d010 - uy) + h[2] * Fy;
    const R t001 = kUnit ? uz + hu * Fz : d001 - om[3] * (d001 - uz) + h[3] * Fz;

    // order 2: off-diagonal toward 0, trace toward rho, deviators toward 0
    const R t110 = d110 - om[4] * (d110 + xy);
    const R t101 = d101 - om[5] * (d101 + xz);
    const R t011 = d011 - om[6] * (d011 + yz);
    const R dtr = d200 + d020 + d002;
    const R dd1 = d200 - d020, dd2 = d200 - d002;
    const R ttr = kUnit ? drho - (ux * ux + uy * uy + uz * uz)
                        : dtr + om[7] * (drho - (ux * ux + uy * uy + uz * uz) - dtr);
    const R td1 = dd1 - om[8] * (dd1 + ux * ux - uy * uy);
    const R td2 = dd2 - om[9] * (dd2 + ux * ux - uz * uz);
    const R t200 = third * (ttr + td1 + td2);
    const R t020 = third * (ttr - R(2) * td1 + td2);
    const R t002 = third * (ttr + td1 - R(2) * td2);

    // order 3: attractors zero (at rate 1 the deviation is -K plus half the source)
    const R s120 = Fxr * k020 + R(2) * Fyr * k110, s102 = Fxr * k002 + R(2) * Fzr * k101;
    const R s210 = R(2) * Fxr * k110 + Fyr * k200, s012 = Fyr * k002 + R(2) * Fzr * k011;
    const R s201 = R(2) * Fxr * k101 + Fzr * k200, s021 = R(2) * Fyr * k011 + Fzr * k020;
    const R s111 = Fxr * k011 + Fyr * k101 + Fzr * k110;
    const R t120 = kUnit ? ux * B + hu * s120 : d120 - om[10] * k120 + h[10] * s120;
    const R t102 = kUnit ? ux * C + hu * s102 : d102 - om[11] * k102 + h[11] * s102;
    const R t210 = kUnit ? A * uy + hu * s210 : d210 - om[12] * k210 + h[12] * s210;
    const R t012 = kUnit ? uy * C + hu * s012 : d012 - om[13] * k012 + h[13] * s012;
    const R t201 = kUnit ? A * uz + hu * s201 : d201 - om[14] * k201 + h[14] * s201;
    const R t021 = kUnit ? B * uz + hu * s021 : d021 - om[15] * k021 + h[15] * s021;
    const R t111 = kUnit ? xy * uz + hu * s111 : d111 - om[16] * k111 + h[16] * s111;

    // full post-collision moments of orders 2-3 (small, or O(1) only through A, B, C)
    const R p110 = xy + t110, p101 = xz + t101, p011 = yz + t011;
    const R p120 = t120 - ux * B, p102 = t102 - ux * C, p210 = t210 - A * uy;
    const R p012 = t012 - uy * C, p201 = t201 - A * uz, p021 = t021 - B * uz;
    const R p111 = t111 - xy * uz;

    // order 4: attractor minus K, with the O(1) products cancelled
    const R M220 = (A * t020 + B * t200 + t200 * t020 + R(2) * p110 * p110 - A * B * drho) * irho;
    const R M202 = (A * t002 + C * t200 + t200 * t002 + R(2) * p101 * p101 - A * C * drho) * irho;
    const R M022 = (B * t002 + C * t020 + t020 * t002 + R(2) * p011 * p011 - B * C * drho) * irho;
    const R M211 = ((A + t200) * p011 + R(2) * p110 * p101) * irho - A * yz;
    const R M121 = ((B + t020) * p101 + R(2) * p110 * p011) * irho - B * xz;
    const R M112 = ((C + t002) * p110 + R(2) * p011 * p101) * irho - C * xy;
    const R s220 = R(2) * (Fxr * k120 + Fyr * k210), s202 = R(2) * (Fxr * k102 + Fzr * k201);
    const R s022 = R(2) * (Fyr * k012 + Fzr * k021);
    const R s211 = R(2) * Fxr * k111 + Fyr * k201 + Fzr * k210;
    const R s121 = Fxr * k021 + R(2) * Fyr * k111 + Fzr * k120;
    const R s112 = Fxr * k012 + Fyr * k102 + R(2) * Fzr * k111;
    const R t220 = kUnit ? M220 + hu * s220 : d220 + om[17] * (M220 - d220) + h[17] * s220;
    const R t202 = kUnit ? M202 + hu * s202 : d202 + om[18] * (M202 - d202) + h[18] * s202;
    const R t022 = kUnit ? M022 + hu * s022 : d022 + om[19] * (M022 - d022) + h[19] * s022;
    const R t211 = kUnit ? M211 + hu * s211 : d211 + om[20] * (M211 - d211) + h[20] * s211;
    const R t121 = kUnit ? M121 + hu * s121 : d121 + om[21] * (M121 - d121) + h[21] * s121;
    const R t112 = kUnit ? M112 + hu * s112 : d112 + om[22] * (M112 - d112) + h[22] * s112;

    // order 5: attractors from post-collision orders 2 and 3 (K_122 = -ux B C, ...)
    const R f25 = R(2.0 / 5.0) * irho;
    const R q200 = A + t200, q020 = B + t020, q002 = C + t002;
    const R M122 = f25 * (q020 * p102 + q002 * p120 + R(4) * p011 * p111
                          + R(2) * (p101 * p021 + p110 * p012)) + ux * B * C;
    const R M212 = f25 * (q200 * p012 + q002 * p210 + R(4) * p101 * p111
                          + R(2) * (p110 * p102 + p011 * p201)) + A * uy * C;
    const R M221 = f25 * (q200 * p021 + q020 * p201 + R(4) * p110 * p111
                          + R(2) * (p011 * p210 + p101 * p120)) + A * B * uz;
    const R s122 = Fxr * k022 + R(2) * (Fyr * k112 + Fzr * k121);
    const R s212 = Fyr * k202 + R(2) * (Fxr * k112 + Fzr * k211);
    const R s221 = Fzr * k220 + R(2) * (Fxr * k121 + Fyr * k211);
    const R t122 = kUnit ? M122 + hu * s122 : d122 + om[23] * (M122 - d122) + h[23] * s122;
    const R t212 = kUnit ? M212 + hu * s212 : d212 + om[24] * (M212 - d212) + h[24] * s212;
    const R t221 = kUnit ? M221 + hu * s221 : d221 + om[25] * (M221 - d221) + h[25] * s221;

    // order 6: attractor from post-collision orders 2 and 4, K_222 = A B C
    const R p112 = C * xy + t112, p121 = B * xz + t121, p211 = A * yz + t211;
    const R M222 = third * irho
                 * (A * t022 + B * t202 + C * t220 + B * C * t200 + A * C * t020 + A * B * t002
                    + t200 * t022 + t020 * t202 + t002 * t220
                    + R(4) * (p110 * p112 + p101 * p121 + p011 * p211) - R(3) * A * B * C * drho);
    const R s222 = R(2) * (Fxr * k122 + Fyr * k212 + Fzr * k221);
    const R t222 = kUnit ? M222 + hu * s222 : d222 + om[26] * (M222 - d222) + h[26] * s222;

    DD(0, 0, 0) = t000; DD(1, 0, 0) = t100; DD(0, 1, 0) = t010; DD(0, 0, 1) = t001;
    DD(1, 1, 0) = t110; DD(1, 0, 1) = t101; DD(0, 1, 1) = t011;
    DD(2, 0, 0) = t200; DD(0, 2, 0) = t020; DD(0, 0, 2) = t002;
    DD(1, 2, 0) = t120; DD(1, 0, 2) = t102; DD(2, 1, 0) = t210; DD(0, 1, 2) = t012;
    DD(2, 0, 1) = t201; DD(0, 2, 1) = t021; DD(1, 1, 1) = t111;
    DD(2, 2, 0) = t220; DD(2, 0, 2) = t202; DD(0, 2, 2) = t022;
    DD(2, 1, 1) = t211; DD(1, 2, 1) = t121; DD(1, 1, 2) = t112;
    DD(1, 2, 2) = t122; DD(2, 1, 2) = t212; DD(2, 2, 1) = t221; DD(2, 2, 2) = t222;
#undef DD
}

// The x sweep split at u: its raw part (independent of u) gives, per x-line (z, y), the sum a+b+c,
// the difference c-a and the sum c+a of the line's links.  The node's density and momentum are
// sums of these nine line values, so the step takes them from here (26 additions instead of 77).
template <class R>
__device__ __forceinline__ void xraw_d3q27(const R f[27], R p[3][3][3])
{
    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        p[e27(a, 2) + 1][e27(a, 1) + 1][e27(a, 0) + 1] = f[a];
    });
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const R a = p[k][j][0], b = p[k][j][1], c = p[k][j][2];
            p[k][j][0] = a + b + c;
            p[k][j][1] = c - a;
            p[k][j][2] = c + a;
        }
}

// One y or z sweep over the nine lines of p: axis 1 sweeps j (lines (k, a)), axis 2 sweeps k
// (lines (j, a)); FP32 pairs the lines at a = 0 and a = 2.
template <bool kInverse, int kAxis, class R>
__device__ __forceinline__ void sweep_yz_d3q27(R p[3][3][3], R u)
{
#define LBM_P(l, m, a) (kAxis == 1 ? p[l][m][a] : p[m][l][a])
    if constexpr (std::is_same<R, float>::value) {
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            float2 v0 = make_float2(LBM_P(l, 0, 0), LBM_P(l, 0, 2));
            float2 v1 = make_float2(LBM_P(l, 1, 0), LBM_P(l, 1, 2));
            float2 v2 = make_float2(LBM_P(l, 2, 0), LBM_P(l, 2, 2));
            if constexpr (kInverse) uncentral_line2(v0, v1, v2, u);
            else central_line2(v0, v1, v2, u);
            LBM_P(l, 0, 0) = v0.x; LBM_P(l, 0, 2) = v0.y;
            LBM_P(l, 1, 0) = v1.x; LBM_P(l, 1, 2) = v1.y;
            LBM_P(l, 2, 0) = v2.x; LBM_P(l, 2, 2) = v2.y;
            if constexpr (kInverse) uncentral_line(LBM_P(l, 0, 1), LBM_P(l, 1, 1), LBM_P(l, 2, 1), u);
            else central_line(LBM_P(l, 0, 1), LBM_P(l, 1, 1), LBM_P(l, 2, 1), u);
        }
    } else {
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if constexpr (kInverse) uncentral_line(LBM_P(l, 0, a), LBM_P(l, 1, a), LBM_P(l, 2, a), u);
                else central_line(LBM_P(l, 0, a), LBM_P(l, 1, a), LBM_P(l, 2, a), u);
            }
    }
#undef LBM_P
}

// Central moments from the raw x-line values: the u part of the x sweep (the same operations as
// central_line), then the y and z sweeps.
template <class R>
__device__ __forceinline__ void central_from_xraw_d3q27(R p[3][3][3], R ux, R uy, R uz)
{
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const R k0 = p[k][j][0], d = p[k][j][1], s = p[k][j][2];
            const R k1 = d - ux * k0;
            p[k][j][1] = k1;
            p[k][j][2] = s - ux * (d + k1);
        }
    sweep_yz_d3q27<false, 1>(p, uy);
    sweep_yz_d3q27<false, 2>(p, uz);
}

// Inverse transform; the populations come out multiplied by 2^L (L = 0 except for FP16 storage,
// whose scale is folded in here instead of at the store).
template <int L = 0, class R>
__device__ __forceinline__ void from_central_d3q27(R p[3][3][3], R f[27], R ux, R uy, R uz)
{
    sweep_yz_d3q27<true, 2>(p, uz);
    sweep_yz_d3q27<true, 1>(p, uy);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) uncentral_line_pow2<L>(p[k][j][0], p[k][j][1], p[k][j][2], ux);
    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        f[a] = p[e27(a, 2) + 1][e27(a, 1) + 1][e27(a, 0) + 1];
    });
}

// Raw moments of a D3Q15 population vector (App. C Step 1), in the moment order of the collision:
// (000, 100, 010, 001, 110, 101, 011, 200, 020, 002, 120, 012, 201, 111, 220).
template <class R>
struct G15Raw {
    R r000, r100, r010, r001, r110, r101, r011, r200, r020, r002, r120, r012, r201, r111, r220;
};

template <class R>
__device__ __forceinline__ G15Raw<R> raw_g_d3q15(const R g[15])
{
    // Axis pairs ...
    const R sx = g[1] + g[2], dx = g[1] - g[2];
    const R sy = g[3] + g[4], dy = g[3] - g[4];
    const R sz = g[5] + g[6], dz = g[5] - g[6];
    // ... and the corner links 7..14 = (+++), (-++), (+-+), (--+), (++-), (-+-), (+--), (---):
    // butterflies over x, then y, then z give sum, x, y, z, xy, xz, yz, xyz weighted sums.
    const R a0 = g[7] + g[8], a1 = g[7] - g[8];     // y+ z+
    const R b0 = g[9] + g[10], b1 = g[9] - g[10];   // y- z+
    const R c0 = g[11] + g[12], c1 = g[11] - g[12]; // y+ z-
    const R d0 = g[13] + g[14], d1 = g[13] - g[14]; // y- z-
    const R zp_s = a0 + b0, zp_y = a0 - b0, zp_x = a1 + b1, zp_xy = a1 - b1;
    const R zm_s = c0 + d0, zm_y = c0 - d0, zm_x = c1 + d1, zm_xy = c1 - d1;
    const R C1 = zp_s + zm_s, Cz = zp_s - zm_s;
    const R Cy = zp_y + zm_y, Cyz = zp_y - zm_y;
    const R Cx = zp_x + zm_x, Cxz = zp_x - zm_x;
    const R Cxy = zp_xy + zm_xy, Cxyz = zp_xy - zm_xy;
    G15Raw<R> r;
    r.r000 = g[0] + sx + sy + sz + C1;
    r.r100 = dx + Cx;
    r.r010 = dy + Cy;
    r.r001 = dz + Cz;
    r.r110 = Cxy;
    r.r101 = Cxz;
    r.r011 = Cyz;
    r.r200 = sx + C1;
    r.r020 = sy + C1;
    r.r002 = sz + C1;
    r.r120 = Cx;
    r.r012 = Cy;
    r.r201 = Cz;
    r.r111 = Cxyz;
    r.r220 = C1;
    return r;
}

// D3Q15 energy collision, App. C Steps 2-5 with option-A attractors (Eq. g-attractorsD3Q15optionA)
// or option B, in deviation form.  `d` holds the Step-1 raw moments of the deviations
// gamma = g - w T_o, and T = T_o + d.r000.  The rest state w T_o has the raw moments
// T_o (1, 1/3, 1/3, 1/3, 1/9) on (000, 200, 020, 002, 220) and none else: they are added before
// Step 2 and removed again after Step 4, so Step 5 writes the post-collision deviations to gd,
// multiplied by 2^L (exactly; L = 10 folds the FP16 storage scale into Step 5's own weights).
template <int L = 0, class R>
__device__ __forceinline__ void collide_g_d3q15(const G15Raw<R>& d, R T_ref, R T, R ux, R uy, R uz,
                                                const R om[15], int gopt, R gd[15])
{
    constexpr double cs2 = 1.0 / 3.0;
    const R rest2 = R(cs2) * T_ref, rest22 = R(1.0 / 9.0) * T_ref;
    const R r000 = T;
    const R r100 = d.r100, r010 = d.r010, r001 = d.r001;
    const R r110 = d.r110, r101 = d.r101, r011 = d.r011;
    const R r200 = d.r200 + rest2, r020 = d.r020 + rest2, r002 = d.r002 + rest2;
    const R r120 = d.r120, r012 = d.r012, r201 = d.r201, r111 = d.r111;
    const R r220 = d.r220 + rest22;

    // Step 2: central moments.
    const R n000 = r000;
    const R n100 = r100 - ux * r000;
    const R n010 = r010 - uy * r000;
    const R n001 = r001 - uz * r000;
    const R n110 = r110 - ux * r010 - uy * n100;
    const R n101 = r101 - ux * r001 - uz * n100;
    const R n011 = r011 - uy * r001 - uz * n010;
    const R n200 = r200 - ux * (r100 + n100);
    const R n020 = r020 - uy * (r010 + n010);
    const R n002 = r002 - uz * (r001 + n001);
    const R n120 = (r120 - uy * (R(2) * r110 - uy * r100)) - ux * n020;
    const R n012 = (r012 - uz * (R(2) * r011 - uz * r010)) - uy * n002;
    const R n201 = (r201 - ux * (R(2) * r101 - ux * r001)) - uz * n200;
    const R n111 = (r111 - ux * r011) - uy * (r101 - ux * r001) - uz * ((r110 - ux * r010) - uy * n100);
    // the raw moment e_x^2 e_y is r012 on D3Q15 (e_x^2 e_y = e_y e_z^2 on every link)
    const R Y1 = r012 - ux * (R(2) * r110 - ux * r010);
    const R Y2 = r220 - ux * (R(2) * r120 - ux * r020);
    const R n220 = Y2 - uy * (R(2) * Y1 - uy * n200);

    // Step 3: relaxation.
    const R t000 = n000 + om[0] * (T - n000);
    const R t100 = n100 - om[1] * n100;
    const R t010 = n010 - om[2] * n010;
    const R t001 = n001 - om[3] * n001;
    const R t110 = n110 - om[4] * n110;
    const R t101 = n101 - om[5] * n101;
    const R t011 = n011 - om[6] * n011;
    const R t200 = n200 + om[7] * (R(cs2) * T - n200);
    const R t020 = n020 + om[8] * (R(cs2) * T - n020);
    const R t002 = n002 + om[9] * (R(cs2) * T - n002);
    // attractors of orders 3-4 from the post-collision moments: option A or option B
    R M120, M012, M201, M111, M220;
    if (gopt == 0) {
        M120 = R(2.0 / 3.0 * cs2) * t100;
        M012 = R(2.0 / 3.0 * cs2) * t010;
        M201 = R(2.0 / 3.0 * cs2) * t001;
        M111 = R(0);
        M220 = R(0.5 * cs2) * (t200 + t020);
    } else {
        const R iT = R(1) / T;
        const R c23 = R(2.0 / 3.0) * iT;
        M120 = c23 * (t020 * t100 + R(2) * t110 * t010);
        M012 = c23 * (t002 * t010 + R(2) * t011 * t001);
        M201 = c23 * (t200 * t001 + R(2) * t101 * t100);
        M111 = c23 * (t110 * t001 + t011 * t100 + t101 * t010);
        M220 = iT * (t200 * t020 + R(2) * t110 * t110);
    }
    const R t120 = n120 + om[10] * (M120 - n120);
    const R t012 = n012 + om[11] * (M012 - n012);
    const R t201 = n201 + om[12] * (M201 - n201);
    const R t111 = n111 + om[13] * (M111 - n111);
    const R t220 = n220 + om[14] * (M220 - n220);

    // Step 4: raw moments from central moments (the inverse of Step 2 in reverse order).
    const R q000 = t000;
    const R q100 = t100 + ux * q000;
    const R q010 = t010 + uy * q000;
    const R q001 = t001 + uz * q000;
    const R q110 = t110 + ux * t010 + uy * q100;
    const R q101 = t101 + ux * t001 + uz * q100;
    const R q011 = t011 + uy * t001 + uz * q010;
    const R q200 = t200 + ux * (t100 + q100);
    const R q020 = t020 + uy * (t010 + q010);
    const R q002 = t002 + uz * (t001 + q001);
    const R q120 = (t120 + uy * (R(2) * t110 + uy * t100)) + ux * q020;
    const R q012 = (t012 + uz * (R(2) * t011 + uz * t010)) + uy * q002;
    const R q201 = (t201 + ux * (R(2) * t101 + ux * t001)) + uz * q200;
    const R q111 = (t111 + ux * t011) + uy * (t101 + ux * t001) + uz * q110;
    const R Z0 = t200;   // the x-central second moment at y-power 0
    const R Z1 = q012 - ux * (R(2) * q110 - ux * q010);
    const R Z2 = t220 + uy * (R(2) * Z1 - uy * Z0);
    const R q220 = Z2 + ux * (R(2) * q120 - ux * q020);

    // Step 5: populations of the deviations (the rest moments removed first).  Axis pairs and the
    // inverse corner transform.
    const R q000d = q000 - T_ref, q200d = q200 - rest2, q020d = q020 - rest2, q002d = q002 - rest2;
    const R q220d = q220 - rest22;
    const R Sx = q200d - q220d, Dx = q100 - q120;
    const R Sy = q020d - q220d, Dy = q010 - q012;
    const R Sz = q002d - q220d, Dz = q001 - q201;
    constexpr double s = double(1ull << L);
    const R g0 = q000d - q200d - q020d - q002d + R(2) * q220d;
    gd[0] = L == 0 ? g0 : R(s) * g0;
    const R hs = R(0.5 * s);
    gd[1] = hs * (Sx + Dx);
    gd[2] = hs * (Sx - Dx);
    gd[3] = hs * (Sy + Dy);
    gd[4] = hs * (Sy - Dy);
    gd[5] = hs * (Sz + Dz);
    gd[6] = hs * (Sz - Dz);
    const R e = R(0.125 * s);
    // z split
    const R P_s = q220d + q201, M_s = q220d - q201;   // sum part for z+ / z-
    const R P_y = q012 + q011, M_y = q012 - q011;
    const R P_x = q120 + q101, M_x = q120 - q101;
    const R P_xy = q110 + q111, M_xy = q110 - q111;
    // y split (z+)
    const R A0 = P_s + P_y, B0 = P_s - P_y, A1 = P_x + P_xy, B1 = P_x - P_xy;
    // y split (z-)
    const R C0 = M_s + M_y, D0 = M_s - M_y, C1_ = M_x + M_xy, D1_ = M_x - M_xy;
    gd[7] = e * (A0 + A1);
    gd[8] = e * (A0 - A1);
    gd[9] = e * (B0 + B1);
    gd[10] = e * (B0 - B1);
    gd[11] = e * (C0 + C1_);
    gd[12] = e * (C0 - C1_);
    gd[13] = e * (D0 + D1_);
    gd[14] = e * (D0 - D1_);
}

// D3Q15 energy collision for the rates lbm_create sets (option A; every rate 1 except those of the
// first-order moments, which carry alpha).  With those rates Step 3 leaves the post-collision
// central moments as T, the relaxed first-order moments t1 = (1 - omega) eta_1, the second-order
// c_s^2 T (diagonal) and 0 (mixed), the third-order (2/3) c_s^2 t1 and 0 (111), and
// eta~_220 = (c_s^2)^2 T: only T and the three first-order raw moments (r100, r010, r001) of the
// pulled populations enter.  Steps 4-5 are those of collide_g_d3q15 with these values (terms that
// vanish dropped), so the output is the same up to rounding; it is written to gd as deviations
// times 2^L.
template <int L = 0, class R>
__device__ __forceinline__ void collide_g_d3q15_unit(R T_ref, R T, R r100, R r010, R r001, R ux,
                                                     R uy, R uz, const R om[15], R gd[15])
{
    constexpr double cs2 = 1.0 / 3.0;
    const R rest2 = R(cs2) * T_ref, rest22 = R(1.0 / 9.0) * T_ref;
    // Steps 2-3: the first-order central moments, relaxed
    const R n100 = r100 - ux * T;
    const R n010 = r010 - uy * T;
    const R n001 = r001 - uz * T;
    const R t100 = n100 - om[1] * n100;
    const R t010 = n010 - om[2] * n010;
    const R t001 = n001 - om[3] * n001;
    const R t2 = R(cs2) * T;                       // t200 = t020 = t002
    const R c3 = R(2.0 / 3.0 * cs2);               // t120 = c3 t100, t012 = c3 t010, t201 = c3 t001
    const R t220 = R(cs2 * cs2) * T;
    // Step 4: raw moments (t110 = t101 = t011 = t111 = 0)
    const R q000 = T;
    const R q100 = t100 + ux * q000;
    const R q010 = t010 + uy * q000;
    const R q001 = t001 + uz * q000;
    const R q110 = ux * t010 + uy * q100;
    const R q101 = ux * t001 + uz * q100;
    const R q011 = uy * t001 + uz * q010;
    const R q200 = t2 + ux * (t100 + q100);
    const R q020 = t2 + uy * (t010 + q010);
    const R q002 = t2 + uz * (t001 + q001);
    const R q120 = (c3 * t100 + uy * (uy * t100)) + ux * q020;
    const R q012 = (c3 * t010 + uz * (uz * t010)) + uy * q002;
    const R q201 = (c3 * t001 + ux * (ux * t001)) + uz * q200;
    const R q111 = uy * (ux * t001) + uz * q110;
    const R Z1 = q012 - ux * (R(2) * q110 - ux * q010);
    const R Z2 = t220 + uy * (R(2) * Z1 - uy * t2);
    const R q220 = Z2 + ux * (R(2) * q120 - ux * q020);
    // Step 5: populations of the deviations
    const R q000d = q000 - T_ref, q200d = q200 - rest2, q020d = q020 - rest2, q002d = q002 - rest2;
    const R q220d = q220 - rest22;
    const R Sx = q200d - q220d, Dx = q100 - q120;
    const R Sy = q020d - q220d, Dy = q010 - q012;
    const R Sz = q002d - q220d, Dz = q001 - q201;
    constexpr double s = double(1ull << L);
    const R g0 = q000d - q200d - q020d - q002d + R(2) * q220d;
    gd[0] = L == 0 ? g0 : R(s) * g0;
    const R hs = R(0.5 * s);
    gd[1] = hs * (Sx + Dx);
    gd[2] = hs * (Sx - Dx);
    gd[3] = hs * (Sy + Dy);
    gd[4] = hs * (Sy - Dy);
    gd[5] = hs * (Sz + Dz);
    gd[6] = hs * (Sz - Dz);
    const R e = R(0.125 * s);
    const R P_s = q220d + q201, M_s = q220d - q201;
    const R P_y = q012 + q011, M_y = q012 - q011;
    const R P_x = q120 + q101, M_x = q120 - q101;
    const R P_xy = q110 + q111, M_xy = q110 - q111;
    const R A0 = P_s + P_y, B0 = P_s - P_y, A1 = P_x + P_xy, B1 = P_x - P_xy;
    const R C0 = M_s + M_y, D0 = M_s - M_y, C1_ = M_x + M_xy, D1_ = M_x - M_xy;
    gd[7] = e * (A0 + A1);
    gd[8] = e * (A0 - A1);
    gd[9] = e * (B0 + B1);
    gd[10] = e * (B0 - B1);
    gd[11] = e * (C0 + C1_);
    gd[12] = e * (C0 - C1_);
    gd[13] = e * (D0 + D1_);
    gd[14] = e * (D0 - D1_);
}

// Zeroth and first raw moments of the D3Q15 deviations (the part of raw_g_d3q15 that the
// unit-rate energy collision needs).
template <class R>
__device__ __forceinline__ void raw01_g_d3q15(const R g[15], R& r000, R& r100, R& r010, R& r001)
{
    const R a0 = g[7] + g[8], a1 = g[7] - g[8];     // y+ z+
    const R b0 = g[9] + g[10], b1 = g[9] - g[10];   // y- z+
    const R c0 = g[11] + g[12], c1 = g[11] - g[12]; // y+ z-
    const R d0 = g[13] + g[14], d1 = g[13] - g[14]; // y- z-
    const R zp_s = a0 + b0, zm_s = c0 + d0;
    const R C1 = zp_s + zm_s, Cz = zp_s - zm_s;
    const R Cy = (a0 - b0) + (c0 - d0);
    const R Cx = (a1 + b1) + (c1 + d1);
    r000 = g[0] + (g[1] + g[2]) + (g[3] + g[4]) + (g[5] + g[6]) + C1;
    r100 = (g[1] - g[2]) + Cx;
    r010 = (g[3] - g[4]) + Cy;
    r001 = (g[5] - g[6]) + Cz;
}

// Macroscopic fields, both collisions and the store of one node whose pulled deviations are in
// f (flow) and g (energy); i is the node's linear index.  kRates (rate_class, checked by the host):
// 0 general rates; 1 the energy rates of lbm_create (collide_g_d3q15_unit); 2 the flow rates of
// lbm_create as well (relax_f_d3q27<true>).
template <class S, class Idx, int kRates = 0>
__device__ __forceinline__ void collide_store_d3q27(typename S::R f[27], typename S::R g[15],
                                                    typename S::T* __restrict__ fout,
                                                    typename S::T* __restrict__ gout,
                                                    const Geometry& geo,
                                                    const Coeffs3D<typename S::R>& c,
                                                    unsigned* status, int i);

template <class S, class Idx, int kRates = 0>
__device__ __forceinline__ void node_step_d3q27(const typename S::T* __restrict__ fin,
                                                const typename S::T* __restrict__ gin,
                                                typename S::T* __restrict__ fout,
                                                typename S::T* __restrict__ gout,
                                                const Geometry& geo, const Coeffs3D<typename S::R>& c,
                                                unsigned* status, int x, int y, int z)
{
    using R = typename S::R;
    const int i = x + geo.nx * y + geo.nxy * z;
    R f[27], g[15];
    // Which pull: decided per warp where possible, so that a warp holding an x-wall node of an
    // interior row runs one x-only pull instead of both the interior and the general pull.
    const bool yz_in = y > 0 && y < geo.ny - 1 && z > 0 && z < geo.nz - 1;
    const bool in = yz_in && x > 0 && x < geo.nx - 1;
    const unsigned lanes = __activemask();
    if (__all_sync(lanes, in)) {
        pull_d3q27_d3q15_interior<S, Idx>(fin, gin, geo, i, c.T_ref, f, g);
    } else if (__all_sync(lanes, yz_in)) {
        const NodeWalls<R> w = node_walls_x<R>(geo, x, y, z);
        pull_d3q27_d3q15<S, Idx>(fin, gin, geo, w, i, c.T_ref, f, g);
    } else if (in) {
        pull_d3q27_d3q15_interior<S, Idx>(fin, gin, geo, i, c.T_ref, f, g);
    } else {
        const NodeWalls<R> w = node_walls<R>(geo, x, y, z, 3);
        pull_d3q27_d3q15<S, Idx>(fin, gin, geo, w, i, c.T_ref, f, g);
    }
    collide_store_d3q27<S, Idx, kRates>(f, g, fout, gout, geo, c, status, i);
}

template <class S, class Idx, int kRates>
__device__ __forceinline__ void collide_store_d3q27(typename S::R f[27], typename S::R g[15],
                                                    typename S::T* __restrict__ fout,
                                                    typename S::T* __restrict__ gout,
                                                    const Geometry& geo,
                                                    const Coeffs3D<typename S::R>& c,
                                                    unsigned* status, int i)
{
    using R = typename S::R;
    // rho = 1 + sum delta, rho u = sum delta e + F/2, T = T_o + sum gamma (the zeroth raw moment of
    // the energy deviations, which the energy collision starts from)
    constexpr bool kUnitG = kRates >= 1, kUnitF = kRates >= 2;
    G15Raw<R> gr;
    R dT;
    if constexpr (kUnitG) raw01_g_d3q15(g, dT, gr.r100, gr.r010, gr.r001);
    else {
        gr = raw_g_d3q15(g);
        dT = gr.r000;
    }
    // Density and momentum: from the raw x-line values for FP16 and FP64 storage, which are bound by
    // the instruction or FP64 rate (51 fewer additions; FP16S +1.2 %); directly from the links for
    // FP32 storage, where keeping the nine line values live adds spills (-0.6 % measured).
    // p[k][j] is the x-line at e_z = k - 1, e_y = j - 1.
    constexpr bool kLineSums = !std::is_same<S, StoreF32>::value;
    R p[3][3][3];
    R drho, jx, jy, jz;
    if constexpr (kLineSums) {
        xraw_d3q27(f, p);
        drho = p[0][0][0];
        jx = p[0][0][1];
#pragma unroll
        for (int l = 1; l < 9; ++l) {
            drho += p[l / 3][l % 3][0];
            jx += p[l / 3][l % 3][1];
        }
        jy = (p[0][2][0] + p[1][2][0] + p[2][2][0]) - (p[0][0][0] + p[1][0][0] + p[2][0][0]);
        jz = (p[2][0][0] + p[2][1][0] + p[2][2][0]) - (p[0][0][0] + p[0][1][0] + p[0][2][0]);
    } else {
        drho = f[0];
        jx = jy = jz = R(0);
        static_for<26>([&](auto A) {
            constexpr int a = decltype(A)::value + 1;
            drho += f[a];
            if (e27(a, 0) == 1) jx += f[a];
            if (e27(a, 0) == -1) jx -= f[a];
            if (e27(a, 1) == 1) jy += f[a];
            if (e27(a, 1) == -1) jy -= f[a];
            if (e27(a, 2) == 1) jz += f[a];
            if (e27(a, 2) == -1) jz -= f[a];
        });
    }
    const R Fb = c.gbeta * dT;
    const R Fx = c.gaxis == 0 ? Fb : R(0);
    const R Fy = c.gaxis == 1 ? Fb : R(0);
    const R Fz = c.gaxis == 2 ? Fb : R(0);
    const R rho = R(1) + drho;
    const R T = c.T_ref + dT;
    const R irho = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * irho;
    const R uy = (jy + R(0.5) * Fy) * irho;
    const R uz = (jz + R(0.5) * Fz) * irho;
    check_node(status, rho, T);

    if constexpr (!kLineSums) xraw_d3q27(f, p);
    central_from_xraw_d3q27(p, ux, uy, uz);
    relax_f_d3q27<kUnitF>(p, drho, irho, ux, uy, uz, Fx, Fy, Fz, c);
    // FP16 storage keeps deviations times 2^10: both collisions return them already scaled
    constexpr bool kF16 = std::is_same<S, StoreF16S>::value;
    constexpr int kL = kF16 ? StoreF16S::kScaleLog2 : 0;
    from_central_d3q27<kL>(p, f, ux, uy, uz);
    // energy collision on the deviations: g receives the post-collision gamma
    if constexpr (kUnitG) collide_g_d3q15_unit<kL>(c.T_ref, T, gr.r100, gr.r010, gr.r001, ux, uy, uz, c.om_g, g);
    else collide_g_d3q15<kL>(gr, c.T_ref, T, ux, uy, uz, c.om_g, c.gopt, g);

    if constexpr (kF16) {
        if (c.fp16_sr) {
            store_node_f16s_sr<27, 15, Idx, true>(fout, gout, (Idx)geo.n, i, f, g);
        } else {
            static_for<27>([&](auto A) {
                constexpr int a = decltype(A)::value;
                StoreF16S::store_scaled(fout, (Idx)a * geo.n + i, f[a]);
            });
            static_for<15>([&](auto B) {
                constexpr int b = decltype(B)::value;
                StoreF16S::store_scaled(gout, (Idx)b * geo.n + i, g[b]);
            });
        }
        return;
    }
    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        S::store_dev(fout, (Idx)a * geo.n + i, f[a], R(w27(a)));
    });
    static_for<15>([&](auto B) {
        constexpr int b = decltype(B)::value;
        S::store_dev(gout, (Idx)b * geo.n + i, g[b], R(w15(b)) * c.T_ref);
    });
}

// Registers per thread of the plain step (sweeps on the 256^3 cavity): FP64 takes what its
// collision needs; FP32 with the reduced collisions of the default rates 72, so that 28 warps fit
// on an SM (+1.0 % against 80; 64 spills and is slower); every other form 80 (24 warps), where 72
// measured slower.
template <class S, int kRates>
struct Launch3D {
    static constexpr int kMaxRegs = sizeof(typename S::R) == 8 ? 255
                                    : (std::is_same<S, StoreF32>::value && kRates == 2 ? 72 : 80);
};

// kRows: each thread updates kRows consecutive rows (y) of its column, one after the other, so a
// block lives kRows times longer and the SM spends a smaller share of its slots on block
// turnover.  The grid's y extent is divided by kRows.
template <class S, class Idx, int kRows = 1, int kRates = 0>
__global__ void __maxnreg__(LBM_MAXREG3D)
    step_d3q27_kernel(const typename S::T* __restrict__ fin, const typename S::T* __restrict__ gin,
                      typename S::T* __restrict__ fout, typename S::T* __restrict__ gout,
                      Geometry geo, Coeffs3D<typename S::R> c, unsigned* status)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * kRows;
    const int z = blockIdx.z;
    if (x >= geo.nx) return;
#pragma unroll 1
    for (int r = 0; r < kRows; ++r) {
        const int y = y0 + r;
        if (y >= geo.ny) return;
        node_step_d3q27<S, Idx, kRates>(fin, gin, fout, gout, geo, c, status, x, y, z);
    }
}

}  // namespace lbm
