// lbm_common.cuh -- storage policies, geometry and the pull-with-walls link for the fused
// collide-and-stream kernels of the Fokker-Planck central-moment LBM (arXiv 2504.09041).
//
// Layout in HBM: structure of arrays, one plane per link, f[a * n + i] with the node index
// i = x + nx * (y + ny * z) (x fastest).  Two buffers per lattice (A -> B, then swap): the
// kernels pull from the post-collision state of the previous step and write the new
// post-collision state at the node itself, so every store is fully coalesced.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>
#include <utility>
#include <type_traits>

namespace lbm {

enum FaceKind { kPeriodic = 0, kAdiabatic = 1, kFixedT = 2 };

// Storage policies: the type in HBM and the type of the moment algebra in registers.  The
// kernels work on deviations from the rest populations (f_a - w_a and g_a - w_a T_o), which keeps
// every quantity of the collision small and resolves it to the register type's precision.
//  - F64 stores the populations themselves and forms the deviation on load.
//  - F32 stores the deviations.
//  - F16S stores the deviations scaled by 2^10, so that deviations down to 6e-8 stay in FP16's
//    normal range (full 11-bit significand) while |deviation| < 64 still fits; the scale is a
//    power of two and adds no rounding.
struct StoreF64 {
    using T = double;
    using R = double;
    __device__ static R load_dev(const T* p, size_t i, R shift) { return __ldg(p + i) - shift; }
    __device__ static void store_dev(T* p, size_t i, R dev, R shift) { p[i] = shift + dev; }
};
// Read-only loads with an L2 prefetch hint of 256 bytes: the pull reads every population plane in
// full, so the sectors around each warp's row are always used by the neighbouring warps.
__device__ __forceinline__ float ldg_pf256(const float* p)
{
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ __half ldg_pf256(const __half* p)
{
    unsigned short v;
    asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __ushort_as_half(v);
}

struct StoreF32 {
    using T = float;
    using R = float;
    __device__ static R load_dev(const T* p, size_t i, R) { return ldg_pf256(p + i); }
    __device__ static void store_dev(T* p, size_t i, R dev, R) { p[i] = dev; }
};
struct StoreF16S {
    using T = __half;
    using R = float;
    static constexpr int kScaleLog2 = 10;
    static constexpr float kScale = 1024.0f;   // 2^kScaleLog2
    static constexpr float kInvScale = 1.0f / 1024.0f;
    __device__ static R load_dev(const T* p, size_t i, R)
    {
        return __half2float(ldg_pf256(p + i)) * kInvScale;
    }
    __device__ static void store_dev(T* p, size_t i, R dev, R) { p[i] = __float2half_rn(dev * kScale); }
    // a deviation already multiplied by kScale
    __device__ static void store_scaled(T* p, size_t i, R scaled) { p[i] = __float2half_rn(scaled); }
    // Two deviations converted together with stochastic rounding: each is rounded up or down to a
    // neighbouring FP16 value with probabilities that make the rounding unbiased, driven by the
    // caller's random bits (Blackwell's cvt.rs).  Returns (half of d0) | (half of d1) << 16.
    __device__ static unsigned pack_sr(R d0, R d1, unsigned rbits)
    {
        return pack_sr_scaled(d0 * kScale, d1 * kScale, rbits);
    }
    // the same for deviations already multiplied by kScale
    __device__ static unsigned pack_sr_scaled(R s0, R s1, unsigned rbits)
    {
        unsigned h2;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(h2) : "f"(s1), "f"(s0), "r"(rbits));
        return h2;
    }
};

// 32-bit integer mix (the "lowbias32" constants of C. Wellons' hash prospector): a counter-style
// source of random bits for stochastic rounding.
__device__ __forceinline__ unsigned mix32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Seed of the stochastic rounding of node i: one full mix of the node index and the FP32 bits of two
// of the node's new values, so the bits are reproducible and change whenever an update below half
// an FP16 step changes the node's state.
__device__ __forceinline__ unsigned sr_seed(unsigned i, float d0, float d1)
{
    return mix32(i * 0x9e3779b9u + (__float_as_uint(d0) ^ (__float_as_uint(d1) << 7)));
}

// Random bits of value pair k of a node: the seed times a distinct odd constant.  Multiplication by
// an odd constant permutes the 32-bit words, so every bit of every pair's word is uniformly
// distributed when the seed is, which is all that unbiased rounding needs.
template <int K>
__device__ __forceinline__ unsigned sr_pair_bits(unsigned seed)
{
    constexpr unsigned mult = 0x9e3779b9u + 2u * (unsigned)K * 0x632be5abu;  // odd for every K
    return seed * mult;
}


// Box geometry and wall description shared by every kernel.
struct Geometry {
    int nx, ny, nz;
    int nxy;                  // nx * ny
    int n;                    // nx * ny * nz (< 2^31)
    int kind[6];              // FaceKind of -x, +x, -y, +y, -z, +z
    double T_wall[6];         // uniform wall temperature of fixed-T faces
    const double* profile[6]; // per-node wall temperature (face tangential order) or nullptr
};

// Relaxation rates and coupling in the register type.
template <class R, int QF, int QG>
struct Coeffs {
    R om_f[QF];   // omega of each relaxed flow moment
    R hf[QF];     // 1 - omega/2 (source weight)
    R om_g[QG];
    R gbeta, T_ref;
    int gaxis;    // 0, 1, 2
    int gopt;     // energy attractors of orders 3-4: 0 = option A, 1 = option B (renormalized)
    int fp16_sr;  // F16S storage: 1 = stochastic rounding of the stored deviations, 0 = nearest
};

// Per-thread wall bookkeeping for the pull.  For an axis, "m" is a link whose source lies at
// coordinate - 1 (component +1) and "p" one whose source lies at coordinate + 1 (component -1).
template <class R>
struct NodeWalls {
    int wrap_m[3], wrap_p[3];   // linear-index correction when a periodic axis wraps
    bool out_m[3], out_p[3];    // the source lies beyond a wall
    bool fix_m[3], fix_p[3];    // ... and that wall has a fixed temperature
    R tw_m[3], tw_p[3];         // wall temperature of that fixed-T face at this node
};

// Wall temperature of face f seen from node (x, y, z).
__device__ __forceinline__ double wall_temperature(const Geometry& g, int f, int x, int y, int z)
{
    const double* p = g.profile[f];
    if (p == nullptr) return g.T_wall[f];
    const int ax = f >> 1;
    const int t = ax == 0 ? y + g.ny * z : (ax == 1 ? x + g.nx * z : x + g.nx * y);
    return __ldg(p + t);
}

template <class R>
__device__ __forceinline__ NodeWalls<R> node_walls(const Geometry& g, int x, int y, int z, int dims)
{
    NodeWalls<R> w;
    const int c[3] = {x, y, z};
    const int ext[3] = {g.nx, g.ny, g.nz};
    const int stride[3] = {1, g.nx, g.nxy};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const bool lo = c[ax] == 0, hi = c[ax] == ext[ax] - 1;
        const bool per = ax >= dims || g.kind[2 * ax] == kPeriodic;
        w.wrap_m[ax] = (lo && per) ? ext[ax] * stride[ax] : 0;
        w.wrap_p[ax] = (hi && per) ? -ext[ax] * stride[ax] : 0;
        w.out_m[ax] = lo && !per;
        w.out_p[ax] = hi && !per;
        w.fix_m[ax] = w.out_m[ax] && g.kind[2 * ax] == kFixedT;
        w.fix_p[ax] = w.out_p[ax] && g.kind[2 * ax + 1] == kFixedT;
        w.tw_m[ax] = w.fix_m[ax] ? R(wall_temperature(g, 2 * ax, x, y, z)) : R(0);
        w.tw_p[ax] = w.fix_p[ax] ? R(wall_temperature(g, 2 * ax + 1, x, y, z)) : R(0);
    }
    return w;
}

// The same bookkeeping for a node whose y and z neighbours all lie inside the box: only the x
// axis can wrap or meet a wall, and the y / z entries are compile-time zeros that fold away.
template <class R>
__device__ __forceinline__ NodeWalls<R> node_walls_x(const Geometry& g, int x, int y, int z)
{
    NodeWalls<R> w;
    const bool lo = x == 0, hi = x == g.nx - 1;
    const bool per = g.kind[0] == kPeriodic;
    w.wrap_m[0] = (lo && per) ? g.nx : 0;
    w.wrap_p[0] = (hi && per) ? -g.nx : 0;
    w.out_m[0] = lo && !per;
    w.out_p[0] = hi && !per;
    w.fix_m[0] = w.out_m[0] && g.kind[0] == kFixedT;
    w.fix_p[0] = w.out_p[0] && g.kind[1] == kFixedT;
    w.tw_m[0] = w.fix_m[0] ? R(wall_temperature(g, 0, x, y, z)) : R(0);
    w.tw_p[0] = w.fix_p[0] ? R(wall_temperature(g, 1, x, y, z)) : R(0);
#pragma unroll
    for (int ax = 1; ax < 3; ++ax) {
        w.wrap_m[ax] = w.wrap_p[ax] = 0;
        w.out_m[ax] = w.out_p[ax] = false;
        w.fix_m[ax] = w.fix_p[ax] = false;
        w.tw_m[ax] = w.tw_p[ax] = R(0);
    }
    return w;
}

// Order of the faces for links that cross two or three walls at an edge or corner of the box:
// the crossed face latest in the order -z, -y, -x, +x, +y, +z (the order of the neighbours'
// linear indices) decides the link's rule.  rank(axis, c) of the face that a link with component
// c = +1 (source at coordinate - 1: the - face) or c = -1 (the + face) crosses on that axis.
__host__ __device__ constexpr int face_rank(int ax, int c)
{
    return c == 1 ? 2 - ax : 3 + ax;
}

// Source of the link arriving at node i along (EX, EY, EZ) after the walls.  Returns the
// linear index of the source node.  *out is set when the source lies beyond a wall.  The crossed
// wall that decides the rule is the one of highest face_rank: *dir is set when it has a fixed
// temperature (anti-bounce-back), and *tw is then its temperature; otherwise the link bounces
// back.  Faces crossed by an edge or corner link therefore decide in the order above.
template <int EX, int EY, int EZ, class R>
__device__ __forceinline__ int link_source(const Geometry& g, const NodeWalls<R>& w, int i,
                                           bool* out, bool* dir, R* tw)
{
    int s = i - (EX + EY * g.nx + EZ * g.nxy);
    bool o = false;
    if (EX == 1) { s += w.wrap_m[0]; o |= w.out_m[0]; }
    if (EX == -1) { s += w.wrap_p[0]; o |= w.out_p[0]; }
    if (EY == 1) { s += w.wrap_m[1]; o |= w.out_m[1]; }
    if (EY == -1) { s += w.wrap_p[1]; o |= w.out_p[1]; }
    if (EZ == 1) { s += w.wrap_m[2]; o |= w.out_m[2]; }
    if (EZ == -1) { s += w.wrap_p[2]; o |= w.out_p[2]; }
    // the deciding face: visit the crossed axes from the highest face rank down
    bool decided = false, d = false;
    R t = R(0);
    constexpr int e[3] = {EX, EY, EZ};
#pragma unroll
    for (int r = 5; r >= 0; --r) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            if (e[ax] == 0 || face_rank(ax, e[ax]) != r) continue;
            const bool crossed = e[ax] == 1 ? w.out_m[ax] : w.out_p[ax];
            const bool fixed = e[ax] == 1 ? w.fix_m[ax] : w.fix_p[ax];
            if (crossed && !decided) {
                decided = true;
                d = fixed;
                t = e[ax] == 1 ? w.tw_m[ax] : w.tw_p[ax];
            }
        }
    }
    *out = o;
    *dir = d;
    *tw = d ? t : R(0);
    return s;
}

// Compile-time loop: calls f(std::integral_constant<int, 0>), ..., f(<N-1>).
template <class F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>)
{
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Store of one node's 2q deviations (flow planes then energy planes) through F16S storage with
// stochastic rounding: consecutive values are converted in pairs.  kScaled: df and dg are already
// multiplied by the storage scale (the seed is still taken from the unscaled values' bits).
template <int QF, int QG, class Idx, bool kScaled = false>
__device__ __forceinline__ void store_node_f16s_sr(__half* __restrict__ fout, __half* __restrict__ gout,
                                                   Idx n, int i, const float* df, const float* dg)
{
    constexpr int Q = QF + QG;
    const float unscale = kScaled ? StoreF16S::kInvScale : 1.0f;
    const unsigned seed = sr_seed((unsigned)i, df[0] * unscale, dg[0] * unscale);
    static_for<(Q + 1) / 2>([&](auto K) {
        constexpr int k = decltype(K)::value;
        constexpr int a0 = 2 * k, a1 = 2 * k + 1;
        // value a of the node: flow plane a, or energy plane a - QF (indices kept in range)
        constexpr int f0 = a0 < QF ? a0 : 0, g0 = a0 < QF ? 0 : a0 - QF;
        constexpr int f1 = a1 < QF ? a1 : 0, g1 = a1 < QF ? 0 : (a1 < Q ? a1 - QF : 0);
        const float v0 = a0 < QF ? df[f0] : dg[g0];
        const float v1 = a1 < Q ? (a1 < QF ? df[f1] : dg[g1]) : 0.0f;
        const unsigned h2 = kScaled ? StoreF16S::pack_sr_scaled(v0, v1, sr_pair_bits<k>(seed))
                                    : StoreF16S::pack_sr(v0, v1, sr_pair_bits<k>(seed));
        const __half h0 = __ushort_as_half((unsigned short)(h2 & 0xffffu));
        const __half h1 = __ushort_as_half((unsigned short)(h2 >> 16));
        if (a0 < QF) fout[(Idx)a0 * n + i] = h0;
        else gout[(Idx)(a0 - QF) * n + i] = h0;
        if (a1 < QF) fout[(Idx)a1 * n + i] = h1;
        else if (a1 < Q) gout[(Idx)(a1 - QF) * n + i] = h1;
    });
}

// Divergence flag: bit 0 set when a node sees a non-finite or non-positive density or a
// non-finite temperature.
template <class R>
__device__ __forceinline__ void check_node(unsigned* status, R rho, R T)
{
    if (!(rho > R(0)) || !(fabs(T) < R(1e30)) || !(rho < R(1e30))) atomicOr(status, 1u);
}

}  // namespace lbm
