// step_d3q27.cuh -- fused pull-stream + FP central-moment collision of the coupled D3Q27 flow
// (Sec. 4.1-4.3) and D3Q15 energy (Appendix C) lattices, one node per thread.
//
// D3Q27: the 27 central moments kappa_abc are produced by three sweeps of 3-link lines (x, y, z),
// which on the tensor-product lattice equals P then F; the inverse sweeps map back.
// D3Q15: raw moments come from the six axis links in pairs and from an 8-point Walsh-Hadamard
// transform of the corner links (the structure of App. C Step 1); the central shift and its exact
// inverse are applied axis by axis (Steps 2 and 4, including the aliased moment 220).
#pragma once

#include "lattices.cuh"
#include "lbm_common.cuh"

namespace lbm {

template <class R>
using Coeffs3D = Coeffs<R, 27, 15>;

// D3Q15 link b for D3Q27 link a, or -1.
__host__ __device__ constexpr int g15_of_27(int a)
{
    return a < 7 ? a : (a >= 19 ? a - 12 : -1);
}

template <class S>
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
        const size_t off = out ? (size_t)o * geo.n + i : (size_t)a * geo.n + s;
        f[a] = S::load(fin, off, R(w27(a)));
        constexpr int b = g15_of_27(a);
        if constexpr (b >= 0) {
            constexpr int ob = opp15(b);
            const size_t og = out ? (size_t)ob * geo.n + i : (size_t)b * geo.n + s;
            const R gv = S::load(gin, og, R(w15(b)) * T_ref);
            g[b] = dir ? R(2.0 * w15(b)) * tw - gv : gv;
        }
    });
}

// Flow collision in central-moment space, K[c][b][a] = kappa_abc (reading R6 of the oracle notes).
// Rate slots follow the moment order of Sec. 4.2; slot 7 is the trace (bulk), slots 8 and 9 the
// deviators kappa_200 - kappa_020 and kappa_200 - kappa_002.
template <class R>
__device__ __forceinline__ void relax_f_d3q27(R K[3][3][3], R rho, R irho, R Fx, R Fy, R Fz,
                                              const Coeffs3D<R>& c)
{
#define KK(a, b, cc) K[cc][b][a]
    const R Fxr = Fx * irho, Fyr = Fy * irho, Fzr = Fz * irho;
    const R* om = c.om_f;
    const R* h = c.hf;

    // orders 0 and 1
    const R t000 = KK(0, 0, 0) + om[0] * (rho - KK(0, 0, 0));
    const R t100 = KK(1, 0, 0) - om[1] * KK(1, 0, 0) + h[1] * Fx;
    const R t010 = KK(0, 1, 0) - om[2] * KK(0, 1, 0) + h[2] * Fy;
    const R t001 = KK(0, 0, 1) - om[3] * KK(0, 0, 1) + h[3] * Fz;

    // order 2
    const R k200 = KK(2, 0, 0), k020 = KK(0, 2, 0), k002 = KK(0, 0, 2);
    const R k110 = KK(1, 1, 0), k101 = KK(1, 0, 1), k011 = KK(0, 1, 1);
    const R t110 = k110 - om[4] * k110;
    const R t101 = k101 - om[5] * k101;
    const R t011 = k011 - om[6] * k011;
    const R tr = k200 + k020 + k002;
    const R d1 = k200 - k020, d2 = k200 - k002;
    const R trt = tr + om[7] * (rho - tr);       // 3 c_s^2 rho = rho
    const R d1t = d1 - om[8] * d1;
    const R d2t = d2 - om[9] * d2;
    const R third = R(1.0 / 3.0);
    const R t200 = third * (trt + d1t + d2t);
    const R t020 = third * (trt - R(2) * d1t + d2t);
    const R t002 = third * (trt + d1t - R(2) * d2t);

    // order 3: attractors zero, sources from the pre-collision moments
    const R k120 = KK(1, 2, 0), k102 = KK(1, 0, 2), k210 = KK(2, 1, 0);
    const R k012 = KK(0, 1, 2), k201 = KK(2, 0, 1), k021 = KK(0, 2, 1), k111 = KK(1, 1, 1);
    const R t120 = k120 - om[10] * k120 + h[10] * (Fxr * k020 + R(2) * Fyr * k110);
    const R t102 = k102 - om[11] * k102 + h[11] * (Fxr * k002 + R(2) * Fzr * k101);
    const R t210 = k210 - om[12] * k210 + h[12] * (R(2) * Fxr * k110 + Fyr * k200);
    const R t012 = k012 - om[13] * k012 + h[13] * (Fyr * k002 + R(2) * Fzr * k011);
    const R t201 = k201 - om[14] * k201 + h[14] * (R(2) * Fxr * k101 + Fzr * k200);
    const R t021 = k021 - om[15] * k021 + h[15] * (R(2) * Fyr * k011 + Fzr * k020);
    const R t111 = k111 - om[16] * k111 + h[16] * (Fxr * k011 + Fyr * k101 + Fzr * k110);

    // order 4: attractors from post-collision order 2
    const R k220 = KK(2, 2, 0), k202 = KK(2, 0, 2), k022 = KK(0, 2, 2);
    const R k211 = KK(2, 1, 1), k121 = KK(1, 2, 1), k112 = KK(1, 1, 2);
    const R M220 = (t200 * t020 + R(2) * t110 * t110) * irho;
    const R M202 = (t200 * t002 + R(2) * t101 * t101) * irho;
    const R M022 = (t020 * t002 + R(2) * t011 * t011) * irho;
    const R M211 = (t200 * t011 + R(2) * t110 * t101) * irho;
    const R M121 = (t020 * t101 + R(2) * t110 * t011) * irho;
    const R M112 = (t002 * t110 + R(2) * t011 * t101) * irho;
    const R t220 = k220 + om[17] * (M220 - k220) + h[17] * R(2) * (Fxr * k120 + Fyr * k210);
    const R t202 = k202 + om[18] * (M202 - k202) + h[18] * R(2) * (Fxr * k102 + Fzr * k201);
    const R t022 = k022 + om[19] * (M022 - k022) + h[19] * R(2) * (Fyr * k012 + Fzr * k021);
    const R t211 = k211 + om[20] * (M211 - k211) + h[20] * (R(2) * Fxr * k111 + Fyr * k201 + Fzr * k210);
    const R t121 = k121 + om[21] * (M121 - k121) + h[21] * (Fxr * k021 + R(2) * Fyr * k111 + Fzr * k120);
    const R t112 = k112 + om[22] * (M112 - k112) + h[22] * (Fxr * k012 + Fyr * k102 + R(2) * Fzr * k111);

    // order 5: attractors from post-collision orders 2 and 3
    const R k122 = KK(1, 2, 2), k212 = KK(2, 1, 2), k221 = KK(2, 2, 1);
    const R two5 = R(2.0 / 5.0) * irho;
    const R M122 = two5 * (t020 * t102 + t002 * t120 + R(4) * t011 * t111
                           + R(2) * (t101 * t021 + t110 * t012));
    const R M212 = two5 * (t200 * t012 + t002 * t210 + R(4) * t101 * t111
                           + R(2) * (t110 * t102 + t011 * t201));
    const R M221 = two5 * (t200 * t021 + t020 * t201 + R(4) * t110 * t111
                           + R(2) * (t011 * t210 + t101 * t120));
    const R t122 = k122 + om[23] * (M122 - k122) + h[23] * (Fxr * k022 + R(2) * (Fyr * k112 + Fzr * k121));
    const R t212 = k212 + om[24] * (M212 - k212) + h[24] * (Fyr * k202 + R(2) * (Fxr * k112 + Fzr * k211));
    const R t221 = k221 + om[25] * (M221 - k221) + h[25] * (Fzr * k220 + R(2) * (Fxr * k121 + Fyr * k211));

    // order 6: attractor from post-collision orders 2 and 4
    const R k222 = KK(2, 2, 2);
    const R M222 = third * irho
                 * (t200 * t022 + t020 * t202 + t002 * t220
                    + R(4) * (t110 * t112 + t101 * t121 + t011 * t211));
    const R t222 = k222 + om[26] * (M222 - k222) + h[26] * R(2) * (Fxr * k122 + Fyr * k212 + Fzr * k221);

    KK(0, 0, 0) = t000; KK(1, 0, 0) = t100; KK(0, 1, 0) = t010; KK(0, 0, 1) = t001;
    KK(1, 1, 0) = t110; KK(1, 0, 1) = t101; KK(0, 1, 1) = t011;
    KK(2, 0, 0) = t200; KK(0, 2, 0) = t020; KK(0, 0, 2) = t002;
    KK(1, 2, 0) = t120; KK(1, 0, 2) = t102; KK(2, 1, 0) = t210; KK(0, 1, 2) = t012;
    KK(2, 0, 1) = t201; KK(0, 2, 1) = t021; KK(1, 1, 1) = t111;
    KK(2, 2, 0) = t220; KK(2, 0, 2) = t202; KK(0, 2, 2) = t022;
    KK(2, 1, 1) = t211; KK(1, 2, 1) = t121; KK(1, 1, 2) = t112;
    KK(1, 2, 2) = t122; KK(2, 1, 2) = t212; KK(2, 2, 1) = t221; KK(2, 2, 2) = t222;
#undef KK
}

template <class R>
__device__ __forceinline__ void to_central_d3q27(const R f[27], R p[3][3][3], R ux, R uy, R uz)
{
    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        p[e27(a, 2) + 1][e27(a, 1) + 1][e27(a, 0) + 1] = f[a];
    });
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) central_line(p[k][j][0], p[k][j][1], p[k][j][2], ux);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) central_line(p[k][0][a], p[k][1][a], p[k][2][a], uy);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) central_line(p[0][b][a], p[1][b][a], p[2][b][a], uz);
}

template <class R>
__device__ __forceinline__ void from_central_d3q27(R p[3][3][3], R f[27], R ux, R uy, R uz)
{
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) uncentral_line(p[0][b][a], p[1][b][a], p[2][b][a], uz);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) uncentral_line(p[k][0][a], p[k][1][a], p[k][2][a], uy);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) uncentral_line(p[k][j][0], p[k][j][1], p[k][j][2], ux);
    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        f[a] = p[e27(a, 2) + 1][e27(a, 1) + 1][e27(a, 0) + 1];
    });
}

// D3Q15 energy collision, App. C Steps 1-5 with option-A attractors (Eq. g-attractorsD3Q15optionA).
// Moment order (000, 100, 010, 001, 110, 101, 011, 200, 020, 002, 120, 012, 201, 111, 220).
template <class R>
__device__ __forceinline__ void collide_g_d3q15(R g[15], R T, R ux, R uy, R uz, const R om[15])
{
    constexpr double cs2 = 1.0 / 3.0;
    // Step 1: raw moments.  Axis pairs ...
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

    const R r000 = g[0] + sx + sy + sz + C1;
    const R r100 = dx + Cx, r010 = dy + Cy, r001 = dz + Cz;
    const R r110 = Cxy, r101 = Cxz, r011 = Cyz;
    const R r200 = sx + C1, r020 = sy + C1, r002 = sz + C1;
    const R r120 = Cx, r012 = Cy, r201 = Cz, r111 = Cxyz, r220 = C1;

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
    const R t120 = n120 + om[10] * (R(2.0 / 3.0 * cs2) * t100 - n120);
    const R t012 = n012 + om[11] * (R(2.0 / 3.0 * cs2) * t010 - n012);
    const R t201 = n201 + om[12] * (R(2.0 / 3.0 * cs2) * t001 - n201);
    const R t111 = n111 - om[13] * n111;
    const R t220 = n220 + om[14] * (R(0.5 * cs2) * (t200 + t020) - n220);

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

    // Step 5: populations.  Axis pairs and the inverse corner transform.
    const R Sx = q200 - q220, Dx = q100 - q120;
    const R Sy = q020 - q220, Dy = q010 - q012;
    const R Sz = q002 - q220, Dz = q001 - q201;
    g[0] = q000 - q200 - q020 - q002 + R(2) * q220;
    g[1] = R(0.5) * (Sx + Dx);
    g[2] = R(0.5) * (Sx - Dx);
    g[3] = R(0.5) * (Sy + Dy);
    g[4] = R(0.5) * (Sy - Dy);
    g[5] = R(0.5) * (Sz + Dz);
    g[6] = R(0.5) * (Sz - Dz);
    const R e = R(0.125);
    // z split
    const R P_s = q220 + q201, M_s = q220 - q201;     // sum part for z+ / z-
    const R P_y = q012 + q011, M_y = q012 - q011;
    const R P_x = q120 + q101, M_x = q120 - q101;
    const R P_xy = q110 + q111, M_xy = q110 - q111;
    // y split (z+)
    const R A0 = P_s + P_y, B0 = P_s - P_y, A1 = P_x + P_xy, B1 = P_x - P_xy;
    // y split (z-)
    const R C0 = M_s + M_y, D0 = M_s - M_y, C1_ = M_x + M_xy, D1_ = M_x - M_xy;
    g[7] = e * (A0 + A1);
    g[8] = e * (A0 - A1);
    g[9] = e * (B0 + B1);
    g[10] = e * (B0 - B1);
    g[11] = e * (C0 + C1_);
    g[12] = e * (C0 - C1_);
    g[13] = e * (D0 + D1_);
    g[14] = e * (D0 - D1_);
}

template <class S>
__device__ __forceinline__ void node_step_d3q27(const typename S::T* __restrict__ fin,
                                                const typename S::T* __restrict__ gin,
                                                typename S::T* __restrict__ fout,
                                                typename S::T* __restrict__ gout,
                                                const Geometry& geo, const Coeffs3D<typename S::R>& c,
                                                unsigned* status, int x, int y, int z)
{
    using R = typename S::R;
    const int i = x + geo.nx * y + geo.nxy * z;
    const NodeWalls<R> w = node_walls<R>(geo, x, y, z, 3);
    R f[27], g[15];
    pull_d3q27_d3q15<S>(fin, gin, geo, w, i, c.T_ref, f, g);

    R T = g[0];
#pragma unroll
    for (int b = 1; b < 15; ++b) T += g[b];
    R rho = f[0], jx = R(0), jy = R(0), jz = R(0);
    static_for<26>([&](auto A) {
        constexpr int a = decltype(A)::value + 1;
        rho += f[a];
        if (e27(a, 0) == 1) jx += f[a];
        if (e27(a, 0) == -1) jx -= f[a];
        if (e27(a, 1) == 1) jy += f[a];
        if (e27(a, 1) == -1) jy -= f[a];
        if (e27(a, 2) == 1) jz += f[a];
        if (e27(a, 2) == -1) jz -= f[a];
    });
    const R Fb = c.gbeta * (T - c.T_ref);
    const R Fx = c.gaxis == 0 ? Fb : R(0);
    const R Fy = c.gaxis == 1 ? Fb : R(0);
    const R Fz = c.gaxis == 2 ? Fb : R(0);
    const R irho = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * irho;
    const R uy = (jy + R(0.5) * Fy) * irho;
    const R uz = (jz + R(0.5) * Fz) * irho;
    check_node(status, rho, T);

    {
        R p[3][3][3];
        to_central_d3q27(f, p, ux, uy, uz);
        relax_f_d3q27(p, rho, irho, Fx, Fy, Fz, c);
        from_central_d3q27(p, f, ux, uy, uz);
    }
    collide_g_d3q15(g, T, ux, uy, uz, c.om_g);

    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        S::store(fout, (size_t)a * geo.n + i, f[a], R(w27(a)));
    });
    static_for<15>([&](auto A) {
        constexpr int b = decltype(A)::value;
        S::store(gout, (size_t)b * geo.n + i, g[b], R(w15(b)) * c.T_ref);
    });
}

template <class S>
struct Launch3D {
    static constexpr int kMinBlocks = sizeof(typename S::R) == 8 ? 1 : 2;
};

template <class S>
__global__ void __launch_bounds__(256, Launch3D<S>::kMinBlocks)
    step_d3q27_kernel(const typename S::T* __restrict__ fin, const typename S::T* __restrict__ gin,
                      typename S::T* __restrict__ fout, typename S::T* __restrict__ gout,
                      Geometry geo, Coeffs3D<typename S::R> c, unsigned* status)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= geo.nx || y >= geo.ny) return;
    node_step_d3q27<S>(fin, gin, fout, gout, geo, c, status, x, y, z);
}

}  // namespace lbm
