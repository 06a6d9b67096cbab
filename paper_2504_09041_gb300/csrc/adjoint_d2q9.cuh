// adjoint_d2q9.cuh -- reverse (adjoint) of the fused D2Q9 flow + D2Q9 energy step.
//
// One forward step maps the post-collision state s_{k-1} to s_k = C(S(s_{k-1}, T_w)): S is the
// streaming with the wall rules (linear in s, affine in the wall temperature through the
// anti-bounce-back), C the per-node collision.  With p_k = S(s_{k-1}) and mu_k = dJ/dp_k,
//   lambda_{k-1} = S^T mu_k              (adjoint streaming: a pull in the opposite direction),
//   mu_{k-1}     = (dC/dp)^T lambda_{k-1} at p_{k-1},
//   dJ/dT_w(j)  += 2 w_a mu_k,a(x)       for every g-link a of wall node x = (j) that takes the
//                                          anti-bounce-back of the design face.
// The fused adjoint kernel does one such step per launch: it gathers lambda at its node from the
// neighbours' mu, recomputes the forward pull and collision of its node from the stored state in
// the adjoint arithmetic type RT, and applies the hand-written vector-Jacobian product of the
// collision.  The design gradient is always accumulated in FP64.
//
// RT is double, float or dfloat (double-float, dfloat.cuh): the VJP is written once with the
// arithmetic operators and instantiated for each.
#pragma once

#include "dfloat.cuh"
#include "step_d2q9.cuh"

namespace lbm {

// Reverse of central_line: outputs (k0, k1, k2) of the line at velocity u with adjoints
// (K0, K1, K2); returns the adjoints (Ab, Bb, Cb) of the inputs and adds d(...)/du to ubar.
template <class RT>
__device__ __forceinline__ void central_line_vjp(RT k0, RT k1, RT u, RT K0, RT K1, RT K2, RT& Ab,
                                                 RT& Bb, RT& Cb, RT& ubar)
{
    const RT d = k1 + u * k0;          // c - a
    const RT K1t = K1 - u * K2;        // total adjoint of k1
    const RT Sb = K2;                  // adjoint of s = c + a
    const RT Db = K1t - u * K2;        // adjoint of d
    const RT K0t = K0 - u * K1t;       // total adjoint of k0
    ubar += -K2 * (d + k1) - K1t * k0;
    Ab = K0t - Db + Sb;
    Bb = K0t;
    Cb = K0t + Db + Sb;
}

// Reverse of uncentral_line: inputs (k0, k1, k2) at velocity u, adjoints (Ab, Bb, Cb) of the
// three links; returns the adjoints of (k0, k1, k2) and adds d(...)/du to ubar.
template <class RT>
__device__ __forceinline__ void uncentral_line_vjp(RT k0, RT k1, RT u, RT Ab, RT Bb, RT Cb, RT& K0,
                                                   RT& K1, RT& K2, RT& ubar)
{
    const RT h = RT(0.5);
    const RT r1 = k1 + u * k0;
    const RT R2 = h * Ab - Bb + h * Cb;
    const RT R1 = -h * Ab + h * Cb + u * R2;
    K2 = R2;
    K1 = u * R2 + R1;
    K0 = Bb + u * R1;
    ubar += R2 * (k1 + r1) + R1 * k0;
}

// Forward sweeps keeping the intermediate values the reverse needs.
template <class RT>
__device__ __forceinline__ void sweeps_fwd(const RT in[9], RT X[3][3], RT D[3][3], RT ux, RT uy)
{
    static_for<9>([&](auto I) {
        constexpr int a = decltype(I)::value;
        X[e9(a, 1) + 1][e9(a, 0) + 1] = in[a];
    });
#pragma unroll
    for (int j = 0; j < 3; ++j) central_line(X[j][0], X[j][1], X[j][2], ux);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) D[j][a] = X[j][a];
#pragma unroll
    for (int a = 0; a < 3; ++a) central_line(D[0][a], D[1][a], D[2][a], uy);
}

// Reverse of sweeps_fwd: adjoints Db of D -> adjoints of the 9 inputs, ux/uy adjoints.
template <class RT>
__device__ __forceinline__ void sweeps_vjp(const RT X[3][3], const RT D[3][3], const RT Db[3][3],
                                           RT ux, RT uy, RT inb[9], RT& uxb, RT& uyb)
{
    RT Xb[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        central_line_vjp(D[0][a], D[1][a], uy, Db[0][a], Db[1][a], Db[2][a], Xb[0][a], Xb[1][a],
                         Xb[2][a], uyb);
    RT Pb[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        central_line_vjp(X[j][0], X[j][1], ux, Xb[j][0], Xb[j][1], Xb[j][2], Pb[j][0], Pb[j][1],
                         Pb[j][2], uxb);
    static_for<9>([&](auto I) {
        constexpr int a = decltype(I)::value;
        inb[a] = Pb[e9(a, 1) + 1][e9(a, 0) + 1];
    });
}

// Forward inverse sweeps keeping the values the reverse needs: T (relaxed moments) -> Y.
template <class RT>
__device__ __forceinline__ void unsweeps_fwd(const RT T[3][3], RT Y[3][3], RT uy)
{
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) Y[j][a] = T[j][a];
#pragma unroll
    for (int a = 0; a < 3; ++a) uncentral_line(Y[0][a], Y[1][a], Y[2][a], uy);
}

// Reverse of the inverse sweeps: adjoints of the 9 outputs -> adjoints Tb of T.
template <class RT>
__device__ __forceinline__ void unsweeps_vjp(const RT T[3][3], const RT Y[3][3], const RT outb[9],
                                             RT ux, RT uy, RT Tb[3][3], RT& uxb, RT& uyb)
{
    RT Ob[3][3];
    static_for<9>([&](auto I) {
        constexpr int a = decltype(I)::value;
        Ob[e9(a, 1) + 1][e9(a, 0) + 1] = outb[a];
    });
    RT Yb[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        uncentral_line_vjp(Y[j][0], Y[j][1], ux, Ob[j][0], Ob[j][1], Ob[j][2], Yb[j][0], Yb[j][1],
                           Yb[j][2], uxb);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        uncentral_line_vjp(T[0][a], T[1][a], uy, Yb[0][a], Yb[1][a], Yb[2][a], Tb[0][a], Tb[1][a],
                           Tb[2][a], uyb);
}

// Reverse of relax_f_d2q9 (deviation form): adjoints tb of the relaxed deviations T -> adjoints
// Db of the pre-collision deviations D and of drho, irho, ux, uy, Fx, Fy.
template <class RT>
__device__ __forceinline__ void relax_f_d2q9_vjp(const RT D[3][3], RT drho, RT irho, RT ux, RT uy,
                                                 RT Fx, RT Fy, const Coeffs2D<RT>& c,
                                                 const RT tb[3][3], RT Db[3][3], RT& drhob,
                                                 RT& irhob, RT& uxb, RT& uyb, RT& Fxb, RT& Fyb)
{
    const RT* o = c.om_f;
    const RT* h = c.hf;
    const RT one = RT(1), two = RT(2), half = RT(0.5), two3 = RT(2.0 / 3.0);
    const RT third = RT(1.0 / 3.0);
    const RT Ax = third + ux * ux, By = third + uy * uy, uxuy = ux * uy;
    const RT D20 = D[0][2], D01 = D[1][0], D11 = D[1][1], D21 = D[1][2];
    const RT D02 = D[2][0], D12 = D[2][1];
    const RT Fxr = Fx * irho, Fyr = Fy * irho;
    const RT k11 = uxuy + D11, k20 = Ax + D20, k02 = By + D02;
    const RT k21 = D21 - Ax * uy, k12 = D12 - ux * By;
    (void)D01;
    // forward values needed by the reverse
    const RT D2s = D20 + D02, D2d = D20 - D02;
    const RT u2s = ux * ux + uy * uy, u2d = ux * ux - uy * uy;
    const RT T2s = D2s + o[3] * (two3 * drho - u2s - D2s);
    const RT T2d = D2d - o[4] * (D2d + u2d);
    const RT T11 = D11 - o[5] * (D11 + uxuy);
    const RT T20 = half * (T2s + T2d), T02 = half * (T2s - T2d);
    const RT t11 = uxuy + T11;
    const RT N = Ax * T02 + By * T20 + T20 * T02 + two * t11 * t11 - Ax * By * drho;

    const RT a00 = tb[0][0], a10 = tb[0][1], a20 = tb[0][2];
    const RT a01 = tb[1][0], a11 = tb[1][1], a21 = tb[1][2];
    const RT a02 = tb[2][0], a12 = tb[2][1], a22 = tb[2][2];
    RT d00 = 0, d10 = 0, d20 = 0, d01 = 0, d11 = 0, d21 = 0, d02 = 0, d12 = 0, d22 = 0;
    RT Axb = 0, Byb = 0, uxuyb = 0, s21b = 0, s12b = 0, s22b = 0;

    // T22 = D22 + o8 (M22 - D22) + h8 s22, M22 = N irho
    d22 += a22 * (one - o[8]);
    const RT M22b = a22 * o[8];
    s22b += a22 * h[8];
    const RT Nb = M22b * irho;
    irhob += M22b * N;
    Axb += Nb * (T02 - By * drho);
    Byb += Nb * (T20 - Ax * drho);
    const RT T02b = a02 + Nb * (Ax + T20);
    const RT T20b = a20 + Nb * (By + T02);
    const RT t11b = Nb * RT(4) * t11;
    drhob += -Nb * Ax * By;
    uxuyb += t11b;
    const RT T11b = a11 + t11b;
    // T12 = D12 - o7 (D12 - ux B) + h7 s12
    d12 += a12 * (one - o[7]);
    uxb += a12 * o[7] * By;
    Byb += a12 * o[7] * ux;
    s12b += a12 * h[7];
    // T21 = D21 - o6 (D21 - A uy) + h6 s21
    d21 += a21 * (one - o[6]);
    Axb += a21 * o[6] * uy;
    uyb += a21 * o[6] * Ax;
    s21b += a21 * h[6];
    // T20, T02 from T2s, T2d
    const RT T2sb = half * (T20b + T02b), T2db = half * (T20b - T02b);
    // T11 = D11 - o5 (D11 + uxuy)
    d11 += T11b * (one - o[5]);
    uxuyb += -T11b * o[5];
    // T2d = D2d - o4 (D2d + u2d); T2s = D2s + o3 (2/3 drho - u2s - D2s)
    const RT D2db = T2db * (one - o[4]);
    const RT u2db = -T2db * o[4];
    const RT D2sb = T2sb * (one - o[3]);
    drhob += T2sb * o[3] * two3;
    const RT u2sb = -T2sb * o[3];
    d20 += D2sb + D2db;
    d02 += D2sb - D2db;
    uxb += two * ux * (u2sb + u2db);
    uyb += two * uy * (u2sb - u2db);
    // T01 = D01 - o2 (D01 - uy) + h2 Fy; T10 = D10 - o1 (D10 - ux) + h1 Fx; T00
    d01 += a01 * (one - o[2]);
    uyb += a01 * o[2];
    Fyb += a01 * h[2];
    d10 += a10 * (one - o[1]);
    uxb += a10 * o[1];
    Fxb += a10 * h[1];
    d00 += a00 * (one - o[0]);
    drhob += a00 * o[0];
    // sources: s21 = 2 Fxr k11 + Fyr k20; s12 = Fxr k02 + 2 Fyr k11; s22 = 2 (Fxr k12 + Fyr k21)
    const RT Fxrb = two * s21b * k11 + s12b * k02 + two * s22b * k12;
    const RT Fyrb = s21b * k20 + two * s12b * k11 + two * s22b * k21;
    const RT k11b = two * s21b * Fxr + two * s12b * Fyr;
    const RT k20b = s21b * Fyr;
    const RT k02b = s12b * Fxr;
    const RT k12b = two * s22b * Fxr;
    const RT k21b = two * s22b * Fyr;
    d12 += k12b;
    uxb += -k12b * By;
    Byb += -k12b * ux;
    d21 += k21b;
    Axb += -k21b * uy;
    uyb += -k21b * Ax;
    Byb += k02b;
    d02 += k02b;
    Axb += k20b;
    d20 += k20b;
    uxuyb += k11b;
    d11 += k11b;
    Fxb += Fxrb * irho;
    Fyb += Fyrb * irho;
    irhob += Fxrb * Fx + Fyrb * Fy;
    uxb += uxuyb * uy + two * ux * Axb;
    uyb += uxuyb * ux + two * uy * Byb;

    Db[0][0] = d00; Db[0][1] = d10; Db[0][2] = d20;
    Db[1][0] = d01; Db[1][1] = d11; Db[1][2] = d21;
    Db[2][0] = d02; Db[2][1] = d12; Db[2][2] = d22;
}

// Reverse of relax_g_d2q9 (full values): adjoints tb of eta~ -> adjoints nb of eta and of T.
// t holds the forward post-collision moments eta~ (needed by the option-B attractors).
template <class RT>
__device__ __forceinline__ void relax_g_d2q9_vjp(const Coeffs2D<RT>& c, const RT t[3][3], RT T,
                                                 const RT tb[3][3], RT nb[3][3], RT& Tb)
{
    const RT* o = c.om_g;
    const RT one = RT(1), half = RT(0.5), two = RT(2);
    const RT cs2 = RT(1.0 / 3.0);
    const RT a00 = tb[0][0], a10 = tb[0][1], a20 = tb[0][2];
    const RT a01 = tb[1][0], a11 = tb[1][1], a21 = tb[1][2];
    const RT a02 = tb[2][0], a12 = tb[2][1], a22 = tb[2][2];
    // t21, t12, t22 = n + o (Mv - n) with attractors from the post-collision lower moments
    const RT n21b = a21 * (one - o[6]), M21b = a21 * o[6];
    const RT n12b = a12 * (one - o[7]), M12b = a12 * o[7];
    const RT n22b = a22 * (one - o[8]), M22b = a22 * o[8];
    RT t10b = a10, t01b = a01, t20b = a20, t02b = a02, t11b = a11;
    if (c.gopt == 0) {
        // Mv21 = (2/3) c_s^2 t01, Mv12 = (2/3) c_s^2 t10, Mv22 = (1/2) c_s^2 (t20 + t02)
        const RT c1 = RT(2.0 / 9.0), c2 = RT(1.0 / 6.0);
        t01b += c1 * M21b;
        t10b += c1 * M12b;
        t20b += c2 * M22b;
        t02b += c2 * M22b;
    } else {
        // Mv21 = c23 (t20 t01 + 2 t11 t10), Mv12 = c23 (t02 t10 + 2 t11 t01),
        // Mv22 = (t20 t02 + 2 t11^2) / T, c23 = 2 / (3 T)
        const RT t10 = t[0][1], t01 = t[1][0], t20 = t[0][2], t02 = t[2][0], t11 = t[1][1];
        const RT iT = one / T, c23 = RT(2.0 / 3.0) * iT;
        const RT P21 = t20 * t01 + two * t11 * t10;
        const RT P12 = t02 * t10 + two * t11 * t01;
        const RT P22 = t20 * t02 + two * t11 * t11;
        const RT g21 = M21b * c23, g12 = M12b * c23, g22 = M22b * iT;
        t20b += g21 * t01 + g22 * t02;
        t02b += g12 * t10 + g22 * t20;
        t01b += g21 * t20 + two * g12 * t11;
        t10b += two * g21 * t11 + g12 * t02;
        t11b += two * (g21 * t10 + g12 * t01) + RT(4) * g22 * t11;
        Tb += -(g21 * P21 + g12 * P12 + g22 * P22) * iT;
    }
    const RT t2sb = half * (t20b + t02b), t2db = half * (t20b - t02b);
    const RT n2sb = t2sb * (one - o[3]);
    Tb += t2sb * o[3] * two * cs2 + a00 * o[0];
    const RT n2db = t2db * (one - o[4]);
    nb[0][0] = a00 * (one - o[0]);
    nb[0][1] = t10b * (one - o[1]);
    nb[1][0] = t01b * (one - o[2]);
    nb[1][1] = t11b * (one - o[5]);
    nb[0][2] = n2sb + n2db;
    nb[2][0] = n2sb - n2db;
    nb[1][2] = n21b;
    nb[2][1] = n12b;
    nb[2][2] = n22b;
}

// Forward values of one node's collision that its vector-Jacobian product needs, computed in the
// register type RF of the forward step (FP32 for FP32 / FP16S states: the same arithmetic the
// forward step applied) and handed to the reverse in RT.
template <class RT>
struct CollideTape {
    RT drho, jx, jy, irho, ux, uy, Fx, Fy, T;
    RT gX[3][3], gN[3][3], gT[3][3], gY[3][3];   // energy: line inputs, central, relaxed, inverse
    RT fX[3][3], fD[3][3], fT[3][3], fY[3][3];   // flow (deviations): the same four stages
};

template <class RF, class RT>
__device__ __forceinline__ void collide_forward_tape(const RF pf[9], const RF pg[9],
                                                     const Coeffs2D<RF>& c, CollideTape<RT>& tp)
{
    const RF half = RF(0.5);
    RF dT = 0, drho = 0, jx = 0, jy = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        dT += pg[a];
        drho += pf[a];
        jx += pf[a] * RF(e9(a, 0));
        jy += pf[a] * RF(e9(a, 1));
    }
    const RF Fb = c.gbeta * dT;
    const RF Fx = c.gaxis == 0 ? Fb : RF(0), Fy = c.gaxis == 1 ? Fb : RF(0);
    const RF rho = RF(1) + drho, irho = RF(1) / rho;
    const RF ux = (jx + half * Fx) * irho, uy = (jy + half * Fy) * irho;
    const RF T = c.T_ref + dT;
    tp.drho = RT(drho); tp.jx = RT(jx); tp.jy = RT(jy); tp.irho = RT(irho);
    tp.ux = RT(ux); tp.uy = RT(uy); tp.Fx = RT(Fx); tp.Fy = RT(Fy); tp.T = RT(T);
    auto keep = [](const RF in[3][3], RT out[3][3]) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int a = 0; a < 3; ++a) out[j][a] = RT(in[j][a]);
    };
    {
        RF gin[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) gin[a] = pg[a] + RF(w9(a)) * c.T_ref;
        RF X[3][3], N[3][3], Tm[3][3], Y[3][3];
        sweeps_fwd(gin, X, N, ux, uy);
        keep(X, tp.gX);
        keep(N, tp.gN);
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int a = 0; a < 3; ++a) Tm[j][a] = N[j][a];
        relax_g_d2q9(Tm, T, c);
        keep(Tm, tp.gT);
        unsweeps_fwd(Tm, Y, uy);
        keep(Y, tp.gY);
    }
    {
        RF X[3][3], D[3][3], Tm[3][3], Y[3][3];
        sweeps_fwd(pf, X, D, ux, uy);
        keep(X, tp.fX);
        keep(D, tp.fD);
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int a = 0; a < 3; ++a) Tm[j][a] = D[j][a];
        relax_f_d2q9(Tm, drho, irho, ux, uy, Fx, Fy, c);
        keep(Tm, tp.fT);
        unsweeps_fwd(Tm, Y, uy);
        keep(Y, tp.fY);
    }
}

// Vector-Jacobian product of the node collision at the forward values tp: adjoints of the
// post-collision deviations (lf, lg) -> adjoints of the pulled deviations (mf, mg), in RT.
template <class RT, bool kSync = false>
__device__ __forceinline__ void collide_vjp_d2q9(const CollideTape<RT>& tp, const RT lf[9],
                                                 const RT lg[9], const Coeffs2D<RT>& c, RT mf[9],
                                                 RT mg[9])
{
    const RT half = RT(0.5);
    const RT drho = tp.drho, jx = tp.jx, jy = tp.jy, irho = tp.irho, ux = tp.ux, uy = tp.uy;
    const RT Fx = tp.Fx, Fy = tp.Fy, T = tp.T;

    RT uxb = 0, uyb = 0, drhob = 0, irhob = 0, Fxb = 0, Fyb = 0, dTb = 0;

    // energy chain: g = w T_ref + gamma -> sweeps -> relax -> inverse sweeps
    {
        RT Tb[3][3], Nb[3][3];
        unsweeps_vjp(tp.gT, tp.gY, lg, ux, uy, Tb, uxb, uyb);
        RT Tfb = 0;
        relax_g_d2q9_vjp(c, tp.gT, T, Tb, Nb, Tfb);
        dTb += Tfb;
        sweeps_vjp(tp.gX, tp.gN, Nb, ux, uy, mg, uxb, uyb);
    }
    if constexpr (kSync) __syncthreads();
    // flow chain on deviations
    {
        RT Tb[3][3], Db[3][3];
        unsweeps_vjp(tp.fT, tp.fY, lf, ux, uy, Tb, uxb, uyb);
        relax_f_d2q9_vjp(tp.fD, drho, irho, ux, uy, Fx, Fy, c, Tb, Db, drhob, irhob, uxb, uyb, Fxb, Fyb);
        sweeps_vjp(tp.fX, tp.fD, Db, ux, uy, mf, uxb, uyb);
    }
    // macroscopic fields: u = (j + F/2) irho, irho = 1 / (1 + drho), F = g beta dT along gravity
    const RT jxb = uxb * irho, jyb = uyb * irho;
    Fxb += half * uxb * irho;
    Fyb += half * uyb * irho;
    irhob += uxb * (jx + half * Fx) + uyb * (jy + half * Fy);
    drhob += -irhob * irho * irho;
    const RT Fbb = (c.gaxis == 0 ? Fxb : RT(0)) + (c.gaxis == 1 ? Fyb : RT(0));
    dTb += c.gbeta * Fbb;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        mf[a] += drhob + jxb * RT(e9(a, 0)) + jyb * RT(e9(a, 1));
        mg[a] += dTb;
    }
}

// First fixed-temperature face crossed by the link arriving along (EX, EY) at a node with walls w
// (the face whose temperature the anti-bounce-back uses), or -1.
template <int EX, int EY, class R>
__device__ __forceinline__ int first_fixed_face(const NodeWalls<R>& w)
{
    if (EX == 1 && w.fix_m[0]) return 0;
    if (EX == -1 && w.fix_p[0]) return 1;
    if (EY == 1 && w.fix_m[1]) return 2;
    if (EY == -1 && w.fix_p[1]) return 3;
    return -1;
}

// One adjoint step at every node (see the file comment).  mu_in = mu_{k+1}, mu_out = mu_k, both
// [18][n] in RT (f links 0..8, then g links 0..8); f_prev, g_prev = s_{k-1} in storage format.
//
// kSync: the block's warps pass a barrier between the phases of the node's work (gather, forward
// tape, energy VJP, flow VJP), so that they run the same stretch of the long unrolled code at the
// same time and share its instruction fetches.  Threads beyond the box then compute on a clamped
// node and store nothing, so every thread reaches every barrier.
template <class S, class RT, bool kSync = false>
__global__ void __launch_bounds__(kSync ? 256 : 128, kSync ? 2 : 1)
    adjoint_step_d2q9_kernel(const typename S::T* __restrict__ f_prev,
                             const typename S::T* __restrict__ g_prev,
                             const RT* __restrict__ mu_in, RT* __restrict__ mu_out, Geometry geo,
                             Coeffs2D<typename S::R> cr, Coeffs2D<RT> c, int design_face,
                             double* __restrict__ grad)
{
    using R = typename S::R;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = x < geo.nx && y < geo.ny;
    if (!kSync && !active) return;
    x = min(x, geo.nx - 1);
    y = min(y, geo.ny - 1);
    const int i = x + geo.nx * y;
    const size_t n = geo.n;
    const NodeWalls<R> w = node_walls<R>(geo, x, y, 0, 2);

    // lambda_{k}(node, b) from mu_{k+1}: the link -b at this node reads its source node + e_b
    RT lf[9], lg[9];
    static_for<9>([&](auto I) {
        constexpr int b = decltype(I)::value;
        constexpr int ob = opp9(b);
        bool out, dir;
        R tw;
        const int s = link_source<e9(ob, 0), e9(ob, 1), 0>(geo, w, i, &out, &dir, &tw);
        if (!out) {
            lf[b] = mu_in[(size_t)b * n + s];
            lg[b] = mu_in[(size_t)(9 + b) * n + s];
        } else {
            lf[b] = mu_in[(size_t)ob * n + i];
            const RT m = mu_in[(size_t)(9 + ob) * n + i];
            lg[b] = dir ? -m : m;
        }
    });

    if constexpr (kSync) __syncthreads();
    // forward pull of p_k from s_{k-1}
    R fr[9], gr[9];
    pull_d2q9<S, size_t>(f_prev, g_prev, geo, w, i, cr.T_ref, fr, gr);
    CollideTape<RT> tape;
    collide_forward_tape(fr, gr, cr, tape);
    if constexpr (kSync) __syncthreads();
    RT mf[9], mg[9];
    collide_vjp_d2q9<RT, kSync>(tape, lf, lg, c, mf, mg);
    if (!active) return;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        mu_out[(size_t)a * n + i] = mf[a];
        mu_out[(size_t)(9 + a) * n + i] = mg[a];
    }

    // design gradient (FP64): anti-bounce-back links of the design face, p = ... + 2 w_a T_w(j)
    double gsum = 0.0;
    bool on_face = false;
    static_for<9>([&](auto I) {
        constexpr int a = decltype(I)::value;
        if (first_fixed_face<e9(a, 0), e9(a, 1)>(w) == design_face) {
            gsum += 2.0 * w9(a) * (double)mg[a];
            on_face = true;
        }
    });
    if (on_face) {
        const int j = design_face < 2 ? y : x;
        grad[j] += gsum;
    }
}

// mu_{n+1} = dJ/dp_{n+1} for J = mean over the objective face of Nu = scale (-8/3 T_w + 3 T_1
// - 1/3 T_2), T_l = T_ref + sum_a p^g_a at the l-th node layer: every g-link of a layer-l node
// gets scale c_l / N (c_1 = 3, c_2 = -1/3); everything else is zero (set beforehand).
template <class RT>
__global__ void adjoint_seed_d2q9_kernel(RT* mu, Geometry geo, int face, double scale)
{
    const int ax = face >> 1, hi = face & 1;
    const int n_face = ax == 0 ? geo.ny : geo.nx;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_face) return;
    const int ext = ax == 0 ? geo.nx : geo.ny;
    for (int l = 0; l < 2; ++l) {
        const int c = hi ? ext - 1 - l : l;
        const int x = ax == 0 ? c : t, y = ax == 0 ? t : c;
        const size_t i = (size_t)x + (size_t)geo.nx * y;
        const double v = scale * (l == 0 ? 3.0 : -1.0 / 3.0) / (double)n_face;
        for (int a = 0; a < 9; ++a) mu[(size_t)(9 + a) * geo.n + i] = (RT)v;
    }
}

}  // namespace lbm
