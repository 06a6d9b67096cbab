// lattices.cuh -- velocity sets, rest weights and the per-axis central-moment transforms.
//
// Velocity sets keep the paper's link order (D2Q9: Eqs. ex, ey; D3Q27: Sec. 5.2; D3Q15:
// Sec. 5.4) so that a population plane a in HBM is the paper's f_a / g_a.
#pragma once

namespace lbm {

// D2Q9 (Eqs. ex, ey).
__host__ __device__ constexpr int e9(int a, int d)
{
    constexpr int t[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                             {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    return t[a][d];
}
__host__ __device__ constexpr int opp9(int a)
{
    constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    return t[a];
}
// Rest populations of the D2Q9 attractors (flow at rho = 1, energy at T = 1).
__host__ __device__ constexpr double w9(int a)
{
    return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// D3Q27 (Sec. 5.2).
__host__ __device__ constexpr int e27(int a, int d)
{
    constexpr int t[27][3] = {
        {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
        {1, 1, 0},   {-1, 1, 0},  {1, -1, 0},  {-1, -1, 0}, {1, 0, 1},   {-1, 0, 1},  {1, 0, -1},
        {-1, 0, -1}, {0, 1, 1},   {0, -1, 1},  {0, 1, -1},  {0, -1, -1}, {1, 1, 1},   {-1, 1, 1},
        {1, -1, 1},  {-1, -1, 1}, {1, 1, -1},  {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};
    return t[a][d];
}
__host__ __device__ constexpr int opp27(int a)
{
    constexpr int t[27] = {0,  2,  1,  4,  3,  6,  5,  10, 9,  8,  7,  14, 13, 12,
                           11, 18, 17, 16, 15, 26, 25, 24, 23, 22, 21, 20, 19};
    return t[a];
}
__host__ __device__ constexpr double w27(int a)
{
    return a == 0 ? 8.0 / 27.0 : (a < 7 ? 2.0 / 27.0 : (a < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
}
// Link index of (ex, ey, ez) in the D3Q27 order.
__host__ __device__ constexpr int idx27(int ex, int ey, int ez)
{
    int r = -1;
    for (int a = 0; a < 27; ++a)
        if (e27(a, 0) == ex && e27(a, 1) == ey && e27(a, 2) == ez) r = a;
    return r;
}

// D3Q15 (Sec. 5.4); its corner links 7..14 are D3Q27 links 19..26 in the same order.
__host__ __device__ constexpr int e15(int a, int d)
{
    constexpr int t[15][3] = {{0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                              {0, 0, 1},   {0, 0, -1}, {1, 1, 1},  {-1, 1, 1},  {1, -1, 1},
                              {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};
    return t[a][d];
}
__host__ __device__ constexpr int opp15(int a)
{
    constexpr int t[15] = {0, 2, 1, 4, 3, 6, 5, 14, 13, 12, 11, 10, 9, 8, 7};
    return t[a];
}
__host__ __device__ constexpr double w15(int a)
{
    return a == 0 ? 2.0 / 9.0 : (a < 7 ? 1.0 / 9.0 : 1.0 / 72.0);
}

// One axis of the central-moment transform on a line of three links with components
// -1, 0, +1 along that axis: (a, b, c) -> (k0, k1, k2) = sum p (e - u)^k, k = 0, 1, 2.
template <class R>
__device__ __forceinline__ void central_line(R& a, R& b, R& c, R u)
{
    const R k0 = a + b + c;
    const R d = c - a;
    const R s = c + a;
    const R k1 = d - u * k0;
    const R k2 = s - u * (d + k1);   // s - 2 u d + u^2 k0
    a = k0;
    b = k1;
    c = k2;
}

// Inverse of central_line: (k0, k1, k2) at velocity u -> the three links (-1, 0, +1).
template <class R>
__device__ __forceinline__ void uncentral_line(R& a, R& b, R& c, R u)
{
    const R k0 = a, k1 = b, k2 = c;
    const R r1 = k1 + u * k0;                 // raw first moment
    const R r2 = k2 + u * (k1 + r1);          // raw second moment: k2 + 2 u k1 + u^2 k0
    const R h = R(0.5);
    a = h * (r2 - r1);
    b = k0 - r2;
    c = h * (r2 + r1);
}

// uncentral_line with its outputs multiplied by 2^L, folded into the line's own halving.  Scaling
// by a power of two is exact, so the outputs are bitwise 2^L times those of uncentral_line.
template <int L, class R>
__device__ __forceinline__ void uncentral_line_pow2(R& a, R& b, R& c, R u)
{
    constexpr double s = double(1ull << L);
    const R k0 = a, k1 = b, k2 = c;
    const R r1 = k1 + u * k0;
    const R r2 = k2 + u * (k1 + r1);
    const R h = R(0.5 * s);
    a = h * (r2 - r1);
    b = L == 0 ? k0 - r2 : R(s) * (k0 - r2);
    c = h * (r2 + r1);
}

// Two lines of one sweep at once, with Blackwell's paired FP32 instructions (FADD2, FFMA2, FMUL2):
// each lane performs exactly the operations of central_line / uncentral_line (a difference c - a
// as the exact fused c + (-1) a).  The sweeps that use them pair the lines at x-orders 0 and 2.
__device__ __forceinline__ void central_line2(float2& a, float2& b, float2& c, float u)
{
    const float2 m1 = make_float2(-1.0f, -1.0f), nu = make_float2(-u, -u);
    const float2 k0 = __fadd2_rn(__fadd2_rn(a, b), c);
    const float2 d = __ffma2_rn(m1, a, c);
    const float2 s = __fadd2_rn(c, a);
    const float2 k1 = __ffma2_rn(nu, k0, d);
    const float2 k2 = __ffma2_rn(nu, __fadd2_rn(d, k1), s);
    a = k0;
    b = k1;
    c = k2;
}

__device__ __forceinline__ void uncentral_line2(float2& a, float2& b, float2& c, float u)
{
    const float2 m1 = make_float2(-1.0f, -1.0f), u2 = make_float2(u, u), h = make_float2(0.5f, 0.5f);
    const float2 k0 = a, k1 = b, k2 = c;
    const float2 r1 = __ffma2_rn(u2, k0, k1);
    const float2 r2 = __ffma2_rn(u2, __fadd2_rn(k1, r1), k2);
    a = __fmul2_rn(h, __ffma2_rn(m1, r1, r2));
    b = __ffma2_rn(m1, r2, k0);
    c = __fmul2_rn(h, __fadd2_rn(r2, r1));
}

}  // namespace lbm
