// aux.cu -- initial state, macroscopic fields, population I/O and the wall Nusselt reduction.
#include "kernels.h"
#include "step_d2q9.cuh"
#include "step_d3q27.cuh"

namespace lbm {

size_t storage_bytes(int prec)
{
    return prec == kF64 ? 8 : (prec == kF32 ? 4 : 2);
}

cudaError_t launch_step(int dim, int prec, const void* fin, const void* gin, void* fout, void* gout,
                        const Geometry& geo, const HostCoeffs& hc, unsigned* status, dim3 block,
                        cudaStream_t st, const TmaMaps* tma)
{
    if (dim == 2) return launch_step_d2q9(prec, fin, gin, fout, gout, geo, hc, status, block, st);
    if (tma && prec == kF32) return launch_step_d3q27_tma_f32(*tma, fin, gin, fout, gout, geo, hc, status, st);
    if (tma && prec == kF16S) return launch_step_d3q27_tma_f16s(*tma, fin, gin, fout, gout, geo, hc, status, st);
    switch (prec) {
    case kF64: return launch_step_d3q27_f64(fin, gin, fout, gout, geo, hc, status, block, st);
    case kF32: return launch_step_d3q27_f32(fin, gin, fout, gout, geo, hc, status, block, st);
    case kF16S: return launch_step_d3q27_f16s(fin, gin, fout, gout, geo, hc, status, block, st);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// Conversions between storage and double (F32 and F16S store deviations from the rest state;
// the full value shift + deviation is formed in double).
// ---------------------------------------------------------------------------------------------
template <class S> struct Conv;
template <> struct Conv<StoreF64> {
    __device__ static double get(const double* p, size_t i, double) { return p[i]; }
    __device__ static void put(double* p, size_t i, double v, double) { p[i] = v; }
};
template <> struct Conv<StoreF32> {
    __device__ static double get(const float* p, size_t i, double s) { return s + (double)p[i]; }
    __device__ static void put(float* p, size_t i, double v, double s) { p[i] = (float)(v - s); }
};
template <> struct Conv<StoreF16S> {
    __device__ static double get(const __half* p, size_t i, double s)
    {
        return s + (double)__half2float(p[i]) * (double)StoreF16S::kInvScale;
    }
    __device__ static void put(__half* p, size_t i, double v, double s)
    {
        p[i] = __double2half((v - s) * (double)StoreF16S::kScale);
    }
};

template <int DIM> struct Lat;
template <> struct Lat<2> {
    static constexpr int QF = 9, QG = 9;
    __device__ static double wf(int a) { return w9(a); }
    __device__ static double wg(int a) { return w9(a); }
};
template <> struct Lat<3> {
    static constexpr int QF = 27, QG = 15;
    __device__ static double wf(int a) { return w27(a); }
    __device__ static double wg(int a) { return w15(a); }
};

// splitmix64 (Steele, Lea and Flood 2014): output i of the stream whose state starts at seed.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Fluid at rest at density 1 and temperature T_init + perturb (2 U_i - 1); the populations are
// the rest attractors (the lattice weights times rho or T).
template <class S, int DIM>
__global__ void init_kernel(typename S::T* f, typename S::T* g, Geometry geo, double T_init,
                            double T_ref, uint64_t seed, double perturb)
{
    using L = Lat<DIM>;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < geo.n;
         i += (long long)gridDim.x * blockDim.x) {
        double T = T_init;
        if (perturb != 0.0) {
            const double u01 = (double)(splitmix64(seed, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
            T += perturb * (2.0 * u01 - 1.0);
        }
        for (int a = 0; a < L::QF; ++a) Conv<S>::put(f, (size_t)a * geo.n + i, L::wf(a), L::wf(a));
        for (int b = 0; b < L::QG; ++b)
            Conv<S>::put(g, (size_t)b * geo.n + i, L::wg(b) * T, L::wg(b) * T_ref);
    }
}

template <class S, int DIM>
__global__ void get_pops_kernel(const typename S::T* f, const typename S::T* g, Geometry geo,
                                double T_ref, double* fo, double* go)
{
    using L = Lat<DIM>;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < geo.n;
         i += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < L::QF; ++a) fo[(size_t)a * geo.n + i] = Conv<S>::get(f, (size_t)a * geo.n + i, L::wf(a));
        for (int b = 0; b < L::QG; ++b)
            go[(size_t)b * geo.n + i] = Conv<S>::get(g, (size_t)b * geo.n + i, L::wg(b) * T_ref);
    }
}

template <class S, int DIM>
__global__ void set_pops_kernel(typename S::T* f, typename S::T* g, Geometry geo, double T_ref,
                                const double* fi, const double* gi)
{
    using L = Lat<DIM>;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < geo.n;
         i += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < L::QF; ++a) Conv<S>::put(f, (size_t)a * geo.n + i, fi[(size_t)a * geo.n + i], L::wf(a));
        for (int b = 0; b < L::QG; ++b)
            Conv<S>::put(g, (size_t)b * geo.n + i, gi[(size_t)b * geo.n + i], L::wg(b) * T_ref);
    }
}

// Streamed populations at one node as deviations from the rest state (the pull of the step
// kernels, without the collision).
template <class S, int DIM>
__device__ __forceinline__ void pulled(const typename S::T* f, const typename S::T* g,
                                       const Geometry& geo, typename S::R T_ref, int x, int y, int z,
                                       typename S::R* fo, typename S::R* go)
{
    using R = typename S::R;
    if constexpr (DIM == 2) {
        const NodeWalls<R> w = node_walls<R>(geo, x, y, 0, 2);
        pull_d2q9<S>(f, g, geo, w, x + geo.nx * y, T_ref, fo, go);
    } else {
        const NodeWalls<R> w = node_walls<R>(geo, x, y, z, 3);
        pull_d3q27_d3q15<S>(f, g, geo, w, x + geo.nx * y + geo.nxy * z, T_ref, fo, go);
    }
}

// Lattice velocity component d of link a.
template <int DIM>
__host__ __device__ constexpr int ev(int a, int d)
{
    if constexpr (DIM == 2) return e9(a, d);
    else return e27(a, d);
}

// rho, u and T at every node (App. A Step 7, App. B Step 7, Sec. 6.1 force); a null output is not
// written.  The sums run over the pulled deviations in the storage's register type (FP32 for FP32
// and FP16 storage, where an FP64 sum made this pass bound by the FP64 pipe) and are promoted to
// FP64 for the outputs.
template <class S, int DIM>
__global__ void fields_kernel(const typename S::T* f, const typename S::T* g, Geometry geo,
                              HostCoeffs hc, double* rho, double* ux, double* uy, double* uz,
                              double* Tout)
{
    using R = typename S::R;
    using L = Lat<DIM>;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < geo.n;
         i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / geo.nxy), rxy = (int)(i - (long long)z * geo.nxy);
        const int y = rxy / geo.nx, x = rxy - y * geo.nx;
        R fo[L::QF], go[L::QG];
        pulled<S, DIM>(f, g, geo, R(hc.T_ref), x, y, z, fo, go);
        R dT = go[0], drho = fo[0], j[3] = {R(0), R(0), R(0)};
        static_for<L::QG - 1>([&](auto B) { dT += go[decltype(B)::value + 1]; });
        static_for<L::QF - 1>([&](auto A) {
            constexpr int a = decltype(A)::value + 1;
            drho += fo[a];
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                if (ev<DIM>(a, d) == 1) j[d] += fo[a];
                if (ev<DIM>(a, d) == -1) j[d] -= fo[a];
            }
        });
        const double T = hc.T_ref + (double)dT, r = 1.0 + (double)drho;
        double F[3] = {0.0, 0.0, 0.0};
        F[hc.gaxis] = hc.gbeta * (double)dT;
        if (rho) rho[i] = r;
        if (ux) ux[i] = ((double)j[0] + 0.5 * F[0]) / r;
        if (uy) uy[i] = ((double)j[1] + 0.5 * F[1]) / r;
        if (uz) uz[i] = ((double)j[2] + 0.5 * F[2]) / r;
        if (Tout) Tout[i] = T;
    }
}

// ---------------------------------------------------------------------------------------------
// Wall Nusselt number (Sec. 6.1): dT/dn = -8/3 T_w + 3 T_1 - 1/3 T_2 from the wall and the first
// two node layers; Nu = scale * dT/dn with scale = -s L / dT.  One thread per wall node, then
// FP64 warp-shuffle reductions of (sum, max with index, min with index), per-block partials and a
// final pass by the last block to finish (deterministic order, ties to the lowest index).
// ---------------------------------------------------------------------------------------------
struct NuAcc {
    double sum, mx, mn;
    int imx, imn;
};

__device__ __forceinline__ void nu_merge(NuAcc& a, const NuAcc& b)
{
    a.sum += b.sum;
    if (b.mx > a.mx || (b.mx == a.mx && b.imx < a.imx)) { a.mx = b.mx; a.imx = b.imx; }
    if (b.mn < a.mn || (b.mn == a.mn && b.imn < a.imn)) { a.mn = b.mn; a.imn = b.imn; }
}

__device__ __forceinline__ NuAcc nu_warp_reduce(NuAcc a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        NuAcc b;
        b.sum = __shfl_down_sync(0xffffffffu, a.sum, o);
        b.mx = __shfl_down_sync(0xffffffffu, a.mx, o);
        b.mn = __shfl_down_sync(0xffffffffu, a.mn, o);
        b.imx = __shfl_down_sync(0xffffffffu, a.imx, o);
        b.imn = __shfl_down_sync(0xffffffffu, a.imn, o);
        nu_merge(a, b);
    }
    return a;
}

__device__ __forceinline__ NuAcc nu_block_reduce(NuAcc a)
{
    __shared__ NuAcc warp_part[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    a = nu_warp_reduce(a);
    if (lane == 0) warp_part[wid] = a;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        NuAcc b = lane < nw ? warp_part[lane]
                            : NuAcc{0.0, -INFINITY, INFINITY, 0x7fffffff, 0x7fffffff};
        a = nu_warp_reduce(b);
    }
    return a;
}

size_t nusselt_scratch_doubles(long n_face)
{
    const long nb = (n_face + 255) / 256;
    return (size_t)(5 * (nb < 1024 ? nb : 1024));
}

template <class S, int DIM>
__global__ void __launch_bounds__(256)
    nusselt_kernel(const typename S::T* f, const typename S::T* g, Geometry geo, double T_ref,
                   int face, int n_face, double scale, double* profile, double* partials,
                   unsigned* ticket, double* result)
{
    using R = typename S::R;
    using L = Lat<DIM>;
    const int ax = face >> 1, hi = face & 1;
    const int ext[3] = {geo.nx, geo.ny, geo.nz};
    NuAcc acc{0.0, -INFINITY, INFINITY, 0x7fffffff, 0x7fffffff};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_face; t += gridDim.x * blockDim.x) {
        int c[3];
        if (ax == 0) { c[1] = t % geo.ny; c[2] = t / geo.ny; }
        if (ax == 1) { c[0] = t % geo.nx; c[2] = t / geo.nx; }
        if (ax == 2) { c[0] = t % geo.nx; c[1] = t / geo.nx; }
        double Tl[2];
        for (int l = 0; l < 2; ++l) {
            c[ax] = hi ? ext[ax] - 1 - l : l;
            R fo[L::QF], go[L::QG];
            pulled<S, DIM>(f, g, geo, R(T_ref), c[0], c[1], c[2], fo, go);
            double s = 0.0;
            for (int b = 0; b < L::QG; ++b) s += (double)go[b];
            Tl[l] = T_ref + s;
        }
        c[ax] = hi ? ext[ax] - 1 : 0;
        const double Tw = wall_temperature(geo, face, c[0], c[1], c[2]);
        const double dTdn = -8.0 / 3.0 * Tw + 3.0 * Tl[0] - 1.0 / 3.0 * Tl[1];
        const double nu = scale * dTdn;
        profile[t] = nu;
        nu_merge(acc, NuAcc{nu, nu, nu, t, t});
    }
    acc = nu_block_reduce(acc);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        double* p = partials + 5 * blockIdx.x;
        p[0] = acc.sum; p[1] = acc.mx; p[2] = (double)acc.imx; p[3] = acc.mn; p[4] = (double)acc.imn;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // Final pass: thread k takes partials k, k + blockDim, ... in order, then a block reduction.
    NuAcc tot{0.0, -INFINITY, INFINITY, 0x7fffffff, 0x7fffffff};
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        const volatile double* p = partials + 5 * k;
        nu_merge(tot, NuAcc{p[0], p[1], p[3], (int)p[2], (int)p[4]});
    }
    tot = nu_block_reduce(tot);
    if (threadIdx.x == 0) {
        result[0] = tot.sum; result[1] = tot.mx; result[2] = (double)tot.imx;
        result[3] = tot.mn; result[4] = (double)tot.imn;
        *ticket = 0u;
    }
}

// ---------------------------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------------------------
static int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    return (int)(b < 65535 ? (b < 1 ? 1 : b) : 65535);
}

#define LBM_DISPATCH(dim, prec, ...)                                                   \
    do {                                                                                \
        if (dim == 2 && prec == kF64) { using S = StoreF64; constexpr int D = 2; __VA_ARGS__; } \
        else if (dim == 2 && prec == kF32) { using S = StoreF32; constexpr int D = 2; __VA_ARGS__; } \
        else if (dim == 2 && prec == kF16S) { using S = StoreF16S; constexpr int D = 2; __VA_ARGS__; } \
        else if (dim == 3 && prec == kF64) { using S = StoreF64; constexpr int D = 3; __VA_ARGS__; } \
        else if (dim == 3 && prec == kF32) { using S = StoreF32; constexpr int D = 3; __VA_ARGS__; } \
        else if (dim == 3 && prec == kF16S) { using S = StoreF16S; constexpr int D = 3; __VA_ARGS__; } \
        else return cudaErrorInvalidValue;                                              \
    } while (0)

cudaError_t launch_init(int dim, int prec, void* f, void* g, const Geometry& geo, double T_init,
                        double T_ref, uint64_t seed, double perturb, cudaStream_t st)
{
    LBM_DISPATCH(dim, prec, {
        using T = typename S::T;
        init_kernel<S, D><<<grid_for(geo.n), 256, 0, st>>>((T*)f, (T*)g, geo, T_init, T_ref, seed,
                                                           perturb);
    });
    return cudaGetLastError();
}

cudaError_t launch_get_pops(int dim, int prec, const void* f, const void* g, const Geometry& geo,
                            double T_ref, double* fo, double* go, cudaStream_t st)
{
    LBM_DISPATCH(dim, prec, {
        using T = typename S::T;
        get_pops_kernel<S, D><<<grid_for(geo.n), 256, 0, st>>>((const T*)f, (const T*)g, geo, T_ref,
                                                               fo, go);
    });
    return cudaGetLastError();
}

cudaError_t launch_set_pops(int dim, int prec, void* f, void* g, const Geometry& geo, double T_ref,
                            const double* fi, const double* gi, cudaStream_t st)
{
    LBM_DISPATCH(dim, prec, {
        using T = typename S::T;
        set_pops_kernel<S, D><<<grid_for(geo.n), 256, 0, st>>>((T*)f, (T*)g, geo, T_ref, fi, gi);
    });
    return cudaGetLastError();
}

cudaError_t launch_fields(int dim, int prec, const void* f, const void* g, const Geometry& geo,
                          const HostCoeffs& hc, double* rho, double* ux, double* uy, double* uz,
                          double* T, cudaStream_t st)
{
    LBM_DISPATCH(dim, prec, {
        using TT = typename S::T;
        fields_kernel<S, D><<<grid_for(geo.n), 256, 0, st>>>((const TT*)f, (const TT*)g, geo, hc, rho,
                                                             ux, uy, uz, T);
    });
    return cudaGetLastError();
}

cudaError_t launch_nusselt(int dim, int prec, const void* f, const void* g, const Geometry& geo,
                           const HostCoeffs& hc, int face, double scale, double* profile,
                           double* scratch, unsigned* ticket, double* result, cudaStream_t st)
{
    const int ax = face >> 1;
    const long n_face = ax == 0 ? (long)geo.ny * geo.nz : (ax == 1 ? (long)geo.nx * geo.nz
                                                                    : (long)geo.nx * geo.ny);
    const int nb = (int)(nusselt_scratch_doubles(n_face) / 5);
    LBM_DISPATCH(dim, prec, {
        using T = typename S::T;
        nusselt_kernel<S, D><<<nb, 256, 0, st>>>((const T*)f, (const T*)g, geo, hc.T_ref, face,
                                                 (int)n_face, scale, profile, scratch, ticket, result);
    });
    return cudaGetLastError();
}

}  // namespace lbm
