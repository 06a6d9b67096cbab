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

#include <type_traits>

#include "dfloat.cuh"
#include "step_d2q9.cuh"

namespace lbm {

// Reverse-mode products multiply an adjoint value (type RT) by a forward value of the node's
// collision (type RF).  The forward values are the forward step's own intermediates: for FP32 /
// FP16 states they are FP32 numbers (RF = float), computed with the same FP32 arithmetic as the
// forward step, and the products, which carry the adjoint, are formed in RT; for FP64 states
// RF = RT.  Quantities that depend on forward values only (the Jacobian's entries) are evaluated
// in RF.
template <class R, class RT>
using TapeT = typename std::conditional<std::is_same<R, float>::value, float, RT>::type;

// adjoint times forward value
template <class RT, class RF>
__device__ __forceinline__ auto am(RT a, RF f)
{
    return a * RT(f);
}
// A double-float adjoint times an FP32 forward value: the leading product with its exact error
// plus the low part's product, left unnormalized for the sum that consumes it (3 flops instead of
// the 4 of a double-float product).
__device__ __forceinline__ dfprod am(dfloat a, float f)
{
    const float p = __fmul_rn(a.hi, f);
    float e = __fmaf_rn(a.hi, f, -p);
    e = __fmaf_rn(a.lo, f, e);
    return dfprod{p, e};
}
__device__ __forceinline__ dfprod am(dfprod a, float f) { return am(dfloat(a), f); }

// x / 2 (exact)
template <class RT>
__device__ __forceinline__ RT halve(RT x)
{
    return x * RT(0.5);
}
__device__ __forceinline__ dfloat halve(dfloat x) { return dfloat(__fmul_rn(0.5f, x.hi), __fmul_rn(0.5f, x.lo)); }

// Reverse of central_line: outputs (k0, k1, k2) of the line at velocity u with adjoints
// (K0, K1, K2); returns the adjoints (Ab, Bb, Cb) of the inputs and adds d(...)/du to ubar.
template <class RT, class RF>
__device__ __forceinline__ void central_line_vjp(RF k0, RF k1, RF u, RT K0, RT K1, RT K2, RT& Ab,
                                                 RT& Bb, RT& Cb, RT& ubar)
{
    const RF d = k1 + u * k0;          // c - a
    const auto uK2 = am(K2, u);
    const RT K1t = K1 - uK2;           // total adjoint of k1
    const RT Db = K1t - uK2;           // adjoint of d; K2 is the adjoint of s = c + a
    const RT K0t = K0 - am(K1t, u);    // total adjoint of k0
    ubar -= am(K2, d + k1) + am(K1t, k0);
    if constexpr (std::is_same<RT, dfloat>::value) {
        const RT P = K0t + K2;     // one double-float sum fewer
        Ab = P - Db;
        Cb = P + Db;
    } else {
        Ab = (K0t - Db) + K2;
        Cb = (K0t + Db) + K2;
    }
    Bb = K0t;
}

// Reverse of uncentral_line: inputs (k0, k1, k2) at velocity u, adjoints (Ab, Bb, Cb) of the
// three links; returns the adjoints of (k0, k1, k2) and adds d(...)/du to ubar.
template <class RT, class RF>
__device__ __forceinline__ void uncentral_line_vjp(RF k0, RF k1, RF u, RT Ab, RT Bb, RT Cb, RT& K0,
                                                   RT& K1, RT& K2, RT& ubar)
{
    const RF r1 = k1 + u * k0;
    const RT hA = halve(Ab), hC = halve(Cb);
    const RT R2 = (hA - Bb) + hC;
    const auto uR2 = am(R2, u);
    const RT R1 = (hC - hA) + uR2;
    K2 = R2;
    K1 = R1 + uR2;
    K0 = Bb + am(R1, u);
    ubar += am(R2, k1 + r1) + am(R1, k0);
}

// Forward sweeps keeping the intermediate values the reverse needs.
template <class R>
__device__ __forceinline__ void sweeps_fwd(const R in[9], R X[3][3], R D[3][3], R ux, R uy)
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
template <class RT, class RF>
__device__ __forceinline__ void sweeps_vjp(const RF X[3][3], const RF D[3][3], const RT Db[3][3],
                                           RF ux, RF uy, RT inb[9], RT& uxb, RT& uyb)
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
template <class R>
__device__ __forceinline__ void unsweeps_fwd(const R T[3][3], R Y[3][3], R uy)
{
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) Y[j][a] = T[j][a];
#pragma unroll
    for (int a = 0; a < 3; ++a) uncentral_line(Y[0][a], Y[1][a], Y[2][a], uy);
}

// Reverse of the inverse sweeps: adjoints of the 9 outputs -> adjoints Tb of T.
template <class RT, class RF>
__device__ __forceinline__ void unsweeps_vjp(const RF T[3][3], const RF Y[3][3], const RT outb[9],
                                             RF ux, RF uy, RT Tb[3][3], RT& uxb, RT& uyb)
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
template <class RT, class RF>
__device__ __forceinline__ void relax_f_d2q9_vjp(const RF D[3][3], RF drho, RF irho, RF ux, RF uy,
                                                 RF Fx, RF Fy, const Coeffs2D<RF>& c,
                                                 const RT tb[3][3], RT Db[3][3], RT& drhob,
                                                 RT& irhob, RT& uxb, RT& uyb, RT& Fxb, RT& Fyb)
{
    const RF* o = c.om_f;
    const RF* h = c.hf;
    const RF one = RF(1), two = RF(2), half = RF(0.5), two3 = RF(2.0 / 3.0);
    const RF third = RF(1.0 / 3.0);
    // forward values (the Jacobian's entries depend on these only)
    const RF Ax = third + ux * ux, By = third + uy * uy, uxuy = ux * uy;
    const RF D20 = D[0][2], D11 = D[1][1], D21 = D[1][2];
    const RF D02 = D[2][0], D12 = D[2][1];
    const RF Fxr = Fx * irho, Fyr = Fy * irho;
    const RF k11 = uxuy + D11, k20 = Ax + D20, k02 = By + D02;
    const RF k21 = D21 - Ax * uy, k12 = D12 - ux * By;
    const RF D2s = D20 + D02, D2d = D20 - D02;
    const RF u2s = ux * ux + uy * uy, u2d = ux * ux - uy * uy;
    const RF T2s = D2s + o[3] * (two3 * drho - u2s - D2s);
    const RF T2d = D2d - o[4] * (D2d + u2d);
    const RF T11 = D11 - o[5] * (D11 + uxuy);
    const RF T20 = half * (T2s + T2d), T02 = half * (T2s - T2d);
    const RF t11 = uxuy + T11;
    const RF N = Ax * T02 + By * T20 + T20 * T02 + two * t11 * t11 - Ax * By * drho;

    const RT a00 = tb[0][0], a10 = tb[0][1], a20 = tb[0][2];
    const RT a01 = tb[1][0], a11 = tb[1][1], a21 = tb[1][2];
    const RT a02 = tb[2][0], a12 = tb[2][1], a22 = tb[2][2];

    // T22 = D22 + o8 (M22 - D22) + h8 s22, M22 = N irho
    const RT d22 = am(a22, one - o[8]);
    const RT M22b = am(a22, o[8]);
    const RT s22b = am(a22, h[8]);
    const RT Nb = am(M22b, irho);
    irhob += am(M22b, N);
    RT Axb = am(Nb, T02 - By * drho);
    RT Byb = am(Nb, T20 - Ax * drho);
    const RT T02b = a02 + am(Nb, Ax + T20);
    const RT T20b = a20 + am(Nb, By + T02);
    const RT t11b = am(Nb, RF(4) * t11);
    drhob -= am(Nb, Ax * By);
    RT uxuyb = t11b;
    const RT T11b = a11 + t11b;
    // T12 = D12 - o7 (D12 - ux B) + h7 s12
    RT d12 = am(a12, one - o[7]);
    uxb += am(a12, o[7] * By);
    Byb += am(a12, o[7] * ux);
    const RT s12b = am(a12, h[7]);
    // T21 = D21 - o6 (D21 - A uy) + h6 s21
    RT d21 = am(a21, one - o[6]);
    Axb += am(a21, o[6] * uy);
    uyb += am(a21, o[6] * Ax);
    const RT s21b = am(a21, h[6]);
    // T20, T02 from T2s, T2d
    const RT T2sb = halve(T20b + T02b), T2db = halve(T20b - T02b);
    // T11 = D11 - o5 (D11 + uxuy)
    RT d11 = am(T11b, one - o[5]);
    uxuyb -= am(T11b, o[5]);
    // T2d = D2d - o4 (D2d + u2d); T2s = D2s + o3 (2/3 drho - u2s - D2s)
    const RT D2db = am(T2db, one - o[4]);
    const RT u2db = -am(T2db, o[4]);
    const RT D2sb = am(T2sb, one - o[3]);
    drhob += am(T2sb, o[3] * two3);
    const RT u2sb = -am(T2sb, o[3]);
    RT d20 = D2sb + D2db;
    RT d02 = D2sb - D2db;
    uxb += am(u2sb + u2db, two * ux);
    uyb += am(u2sb - u2db, two * uy);
    // T01 = D01 - o2 (D01 - uy) + h2 Fy; T10 = D10 - o1 (D10 - ux) + h1 Fx; T00
    const RT d01 = am(a01, one - o[2]);
    uyb += am(a01, o[2]);
    Fyb += am(a01, h[2]);
    const RT d10 = am(a10, one - o[1]);
    uxb += am(a10, o[1]);
    Fxb += am(a10, h[1]);
    const RT d00 = am(a00, one - o[0]);
    drhob += am(a00, o[0]);
    // sources: s21 = 2 Fxr k11 + Fyr k20; s12 = Fxr k02 + 2 Fyr k11; s22 = 2 (Fxr k12 + Fyr k21)
    const RT Fxrb = am(s21b, two * k11) + am(s12b, k02) + am(s22b, two * k12);
    const RT Fyrb = am(s21b, k20) + am(s12b, two * k11) + am(s22b, two * k21);
    const RT k11b = am(s21b, two * Fxr) + am(s12b, two * Fyr);
    const RT k20b = am(s21b, Fyr);
    const RT k02b = am(s12b, Fxr);
    const RT k12b = am(s22b, two * Fxr);
    const RT k21b = am(s22b, two * Fyr);
    d12 += k12b;
    uxb -= am(k12b, By);
    Byb -= am(k12b, ux);
    d21 += k21b;
    Axb -= am(k21b, uy);
    uyb -= am(k21b, Ax);
    Byb += k02b;
    d02 += k02b;
    Axb += k20b;
    d20 += k20b;
    uxuyb += k11b;
    d11 += k11b;
    Fxb += am(Fxrb, irho);
    Fyb += am(Fyrb, irho);
    irhob += am(Fxrb, Fx) + am(Fyrb, Fy);
    uxb += am(uxuyb, uy) + am(Axb, two * ux);
    uyb += am(uxuyb, ux) + am(Byb, two * uy);

    Db[0][0] = d00; Db[0][1] = d10; Db[0][2] = d20;
    Db[1][0] = d01; Db[1][1] = d11; Db[1][2] = d21;
    Db[2][0] = d02; Db[2][1] = d12; Db[2][2] = d22;
}

// Reverse of relax_g_d2q9 (full values): adjoints tb of eta~ -> adjoints nb of eta and of T.
// t holds the forward post-collision moments eta~ (needed by the option-B attractors).
template <class RT, class RF>
__device__ __forceinline__ void relax_g_d2q9_vjp(const Coeffs2D<RF>& c, const RF t[3][3], RF T,
                                                 const RT tb[3][3], RT nb[3][3], RT& Tb)
{
    const RF* o = c.om_g;
    const RF one = RF(1), two = RF(2);
    const RF cs2 = RF(1.0 / 3.0);
    const RT a00 = tb[0][0], a10 = tb[0][1], a20 = tb[0][2];
    const RT a01 = tb[1][0], a11 = tb[1][1], a21 = tb[1][2];
    const RT a02 = tb[2][0], a12 = tb[2][1], a22 = tb[2][2];
    // t21, t12, t22 = n + o (Mv - n) with attractors from the post-collision lower moments
    const RT n21b = am(a21, one - o[6]), M21b = am(a21, o[6]);
    const RT n12b = am(a12, one - o[7]), M12b = am(a12, o[7]);
    const RT n22b = am(a22, one - o[8]), M22b = am(a22, o[8]);
    RT t10b = a10, t01b = a01, t20b = a20, t02b = a02, t11b = a11;
    if (c.gopt == 0) {
        // Mv21 = (2/3) c_s^2 t01, Mv12 = (2/3) c_s^2 t10, Mv22 = (1/2) c_s^2 (t20 + t02)
        const RF c1 = RF(2.0 / 9.0), c2 = RF(1.0 / 6.0);
        t01b += am(M21b, c1);
        t10b += am(M12b, c1);
        t20b += am(M22b, c2);
        t02b += am(M22b, c2);
    } else {
        // Mv21 = c23 (t20 t01 + 2 t11 t10), Mv12 = c23 (t02 t10 + 2 t11 t01),
        // Mv22 = (t20 t02 + 2 t11^2) / T, c23 = 2 / (3 T)
        const RF t10 = t[0][1], t01 = t[1][0], t20 = t[0][2], t02 = t[2][0], t11 = t[1][1];
        const RF iT = one / T, c23 = RF(2.0 / 3.0) * iT;
        const RF P21 = t20 * t01 + two * t11 * t10;
        const RF P12 = t02 * t10 + two * t11 * t01;
        const RF P22 = t20 * t02 + two * t11 * t11;
        const RT g21 = am(M21b, c23), g12 = am(M12b, c23), g22 = am(M22b, iT);
        t20b += am(g21, t01) + am(g22, t02);
        t02b += am(g12, t10) + am(g22, t20);
        t01b += am(g21, t20) + am(g12, two * t11);
        t10b += am(g21, two * t11) + am(g12, t02);
        t11b += am(g21, two * t10) + am(g12, two * t01);
        t11b += am(g22, RF(4) * t11);
        const RT Pb = am(g21, P21) + am(g12, P12);
        Tb -= am(Pb + am(g22, P22), iT);
    }
    const RT t2sb = halve(t20b + t02b), t2db = halve(t20b - t02b);
    const RT n2sb = am(t2sb, one - o[3]);
    Tb += am(t2sb, o[3] * two * cs2) + am(a00, o[0]);
    const RT n2db = am(t2db, one - o[4]);
    nb[0][0] = am(a00, one - o[0]);
    nb[0][1] = am(t10b, one - o[1]);
    nb[1][0] = am(t01b, one - o[2]);
    nb[1][1] = am(t11b, one - o[5]);
    nb[0][2] = n2sb + n2db;
    nb[2][0] = n2sb - n2db;
    nb[1][2] = n21b;
    nb[2][1] = n12b;
    nb[2][2] = n22b;
}

// Forward values of one node's collision that its vector-Jacobian product needs, computed in the
// register type R of the forward step (FP32 for FP32 / FP16S states: the same arithmetic the
// forward step applied) and kept in RF (TapeT: R itself for FP32 states, the adjoint type for
// FP64 states).
template <class RF>
struct CollideTape {
    RF drho, jx, jy, irho, ux, uy, Fx, Fy, T;
    RF gX[3][3], gN[3][3], gT[3][3], gY[3][3];   // energy: line inputs, central, relaxed, inverse
    RF fX[3][3], fD[3][3], fT[3][3], fY[3][3];   // flow (deviations): the same four stages
};

template <class R, class RF>
__device__ __forceinline__ void collide_forward_tape(const R pf[9], const R pg[9],
                                                     const Coeffs2D<R>& c, CollideTape<RF>& tp)
{
    const R half = R(0.5);
    R dT = 0, drho = 0, jx = 0, jy = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        dT += pg[a];
        drho += pf[a];
        jx += pf[a] * R(e9(a, 0));
        jy += pf[a] * R(e9(a, 1));
    }
    const R Fb = c.gbeta * dT;
    const R Fx = c.gaxis == 0 ? Fb : R(0), Fy = c.gaxis == 1 ? Fb : R(0);
    const R rho = R(1) + drho, irho = R(1) / rho;
    const R ux = (jx + half * Fx) * irho, uy = (jy + half * Fy) * irho;
    const R T = c.T_ref + dT;
    tp.drho = RF(drho); tp.jx = RF(jx); tp.jy = RF(jy); tp.irho = RF(irho);
    tp.ux = RF(ux); tp.uy = RF(uy); tp.Fx = RF(Fx); tp.Fy = RF(Fy); tp.T = RF(T);
    auto keep = [](const R in[3][3], RF out[3][3]) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int a = 0; a < 3; ++a) out[j][a] = RF(in[j][a]);
    };
    {
        R gin[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) gin[a] = pg[a] + R(w9(a)) * c.T_ref;
        R X[3][3], N[3][3], Tm[3][3], Y[3][3];
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
        R X[3][3], D[3][3], Tm[3][3], Y[3][3];
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
// kSync: a block-wide barrier between the energy and the flow products (see the kernel).
template <class RT, class RF, bool kSync = false>
__device__ __forceinline__ void collide_vjp_d2q9(const CollideTape<RF>& tp, const RT lf[9],
                                                 const RT lg[9], const Coeffs2D<RF>& c, RT mf[9],
                                                 RT mg[9])
{
    const RF half = RF(0.5);
    const RF drho = tp.drho, jx = tp.jx, jy = tp.jy, irho = tp.irho, ux = tp.ux, uy = tp.uy;
    const RF Fx = tp.Fx, Fy = tp.Fy, T = tp.T;

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
    const RT jxb = am(uxb, irho), jyb = am(uyb, irho);
    Fxb += am(uxb, half * irho);
    Fyb += am(uyb, half * irho);
    irhob += am(uxb, jx + half * Fx) + am(uyb, jy + half * Fy);
    drhob -= am(irhob, irho * irho);
    const RT Fbb = c.gaxis == 0 ? Fxb : (c.gaxis == 1 ? Fyb : RT(0));
    dTb += am(Fbb, c.gbeta);
    static_for<9>([&](auto I) {
        constexpr int a = decltype(I)::value;
        RT m = drhob;
        if constexpr (e9(a, 0) == 1) m += jxb;
        if constexpr (e9(a, 0) == -1) m -= jxb;
        if constexpr (e9(a, 1) == 1) m += jyb;
        if constexpr (e9(a, 1) == -1) m -= jyb;
        mf[a] += m;
        mg[a] += dTb;
    });
}

// The fixed-temperature face whose anti-bounce-back the link arriving along (EX, EY) at a node
// with walls w takes (the crossed face of highest face_rank, when it is a fixed-T face), or -1.
template <int EX, int EY, class R>
__device__ __forceinline__ int first_fixed_face(const NodeWalls<R>& w)
{
    const bool cx = EX == 1 ? w.out_m[0] : (EX == -1 ? w.out_p[0] : false);
    const bool cy = EY == 1 ? w.out_m[1] : (EY == -1 ? w.out_p[1] : false);
    const int fx = EX == 1 ? 0 : 1, fy = EY == 1 ? 2 : 3;
    const bool fix_x = EX == 1 ? w.fix_m[0] : (EX == -1 ? w.fix_p[0] : false);
    const bool fix_y = EY == 1 ? w.fix_m[1] : (EY == -1 ? w.fix_p[1] : false);
    // the y face outranks the x face for EY = -1 (the +y face); the x face outranks -y
    const bool y_first = EY == -1;
    if (y_first && cy) return fix_y ? fy : -1;
    if (cx) return fix_x ? fx : -1;
    if (cy) return fix_y ? fy : -1;
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
                             Coeffs2D<typename S::R> cr, Coeffs2D<TapeT<typename S::R, RT>> c,
                             int design_face, double* __restrict__ grad)
{
    using R = typename S::R;
    using RF = TapeT<R, RT>;
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
    CollideTape<RF> tape;
    collide_forward_tape(fr, gr, cr, tape);
    if constexpr (kSync) __syncthreads();
    RT mf[9], mg[9];
    collide_vjp_d2q9<RT, RF, kSync>(tape, lf, lg, c, mf, mg);
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
