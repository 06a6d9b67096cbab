// noalloc.cu -- the wall Nusselt reduction for callers that cannot allocate device memory.
//
// lbm_nusselt_static() reads energy populations from a buffer the caller owns and writes its
// result into another buffer the caller owns.  The only other memory it needs -- one partial
// result per thread block and the "last block" ticket -- lives in the fixed device array below,
// so the call itself never allocates.  The array belongs to this library image: every GPU that
// loads the library holds it (about 160 KB) until the process exits.
#include <climits>
#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"
#include "kernels.h"
#include "lattices.cuh"
#include "lbm_common.cuh"

namespace lbm {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = LBM_NUSSELT_STATIC_MAX_FACE_NODES / kThreads;

// Scratch: kMaxBlocks partials of 5 doubles, then the ticket (kept as a double-sized slot).
static __device__ __align__(256) double g_scratch[5 * kMaxBlocks + 1];

struct Acc {
    double sum, mx, mn;
    int imx, imn;
};

__device__ __forceinline__ void merge(Acc& a, const Acc& b)
{
    a.sum += b.sum;
    if (b.mx > a.mx || (b.mx == a.mx && b.imx < a.imx)) { a.mx = b.mx; a.imx = b.imx; }
    if (b.mn < a.mn || (b.mn == a.mn && b.imn < a.imn)) { a.mn = b.mn; a.imn = b.imn; }
}

__device__ __forceinline__ Acc warp_reduce(Acc a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Acc b;
        b.sum = __shfl_down_sync(0xffffffffu, a.sum, o);
        b.mx = __shfl_down_sync(0xffffffffu, a.mx, o);
        b.mn = __shfl_down_sync(0xffffffffu, a.mn, o);
        b.imx = __shfl_down_sync(0xffffffffu, a.imx, o);
        b.imn = __shfl_down_sync(0xffffffffu, a.imn, o);
        merge(a, b);
    }
    return a;
}

__device__ __forceinline__ Acc block_reduce(Acc a)
{
    __shared__ Acc part[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    a = warp_reduce(a);
    if (lane == 0) part[wid] = a;
    __syncthreads();
    if (wid == 0) {
        Acc b = lane < kThreads / 32 ? part[lane] : Acc{0.0, -INFINITY, INFINITY, 0x7fffffff, 0x7fffffff};
        a = warp_reduce(b);
    }
    return a;
}

// Temperature of the streamed energy populations at one node: sum over the links of the pulled
// g with the wall rules (bounce-back, anti-bounce-back at T_wall).
template <class S, int DIM>
__device__ __forceinline__ double pulled_T(const typename S::T* g, const Geometry& geo, double T_ref,
                                           int x, int y, int z)
{
    using R = typename S::R;
    const NodeWalls<R> w = node_walls<R>(geo, x, y, z, DIM);
    const int i = x + geo.nx * y + geo.nxy * z;
    double sum = 0.0;   // deviations summed first, then T_ref added (the order of lbm_nusselt)
    if constexpr (DIM == 2) {
        static_for<9>([&](auto A) {
            constexpr int a = decltype(A)::value;
            bool out, dir;
            R tw;
            const int s = link_source<e9(a, 0), e9(a, 1), 0>(geo, w, i, &out, &dir, &tw);
            const size_t off = out ? (size_t)opp9(a) * geo.n + i : (size_t)a * geo.n + s;
            const R gv = S::load_dev(g, off, R(w9(a)) * R(T_ref));
            sum += (double)(dir ? R(2.0 * w9(a)) * (tw - R(T_ref)) - gv : gv);
        });
    } else {
        static_for<15>([&](auto B) {
            constexpr int b = decltype(B)::value;
            bool out, dir;
            R tw;
            const int s = link_source<e15(b, 0), e15(b, 1), e15(b, 2)>(geo, w, i, &out, &dir, &tw);
            const size_t off = out ? (size_t)opp15(b) * geo.n + i : (size_t)b * geo.n + s;
            const R gv = S::load_dev(g, off, R(w15(b)) * R(T_ref));
            sum += (double)(dir ? R(2.0 * w15(b)) * (tw - R(T_ref)) - gv : gv);
        });
    }
    return T_ref + sum;
}

// One thread per wall node, one partial per block in scratch[], the last block finishes.
template <class S, int DIM>
__global__ void __launch_bounds__(kThreads)
    nusselt_static_kernel(const typename S::T* g, Geometry geo, double T_ref, int face, int n_face,
                          double scale, double* scratch, double* result)
{
    const int ax = face >> 1, hi = face & 1;
    const int ext[3] = {geo.nx, geo.ny, geo.nz};
    Acc acc{0.0, -INFINITY, INFINITY, 0x7fffffff, 0x7fffffff};
    const int t = blockIdx.x * kThreads + threadIdx.x;
    if (t < n_face) {
        int c[3];
        if (ax == 0) { c[1] = t % geo.ny; c[2] = t / geo.ny; }
        if (ax == 1) { c[0] = t % geo.nx; c[2] = t / geo.nx; }
        if (ax == 2) { c[0] = t % geo.nx; c[1] = t / geo.nx; }
        double Tl[2];
        for (int l = 0; l < 2; ++l) {
            c[ax] = hi ? ext[ax] - 1 - l : l;
            Tl[l] = pulled_T<S, DIM>(g, geo, T_ref, c[0], c[1], c[2]);
        }
        const double Tw = geo.T_wall[face];
        const double nu = scale * (-8.0 / 3.0 * Tw + 3.0 * Tl[0] - 1.0 / 3.0 * Tl[1]);
        acc = Acc{nu, nu, nu, t, t};
    }
    acc = block_reduce(acc);
    unsigned* ticket = reinterpret_cast<unsigned*>(scratch + 5 * kMaxBlocks);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        double* p = scratch + 5 * blockIdx.x;
        p[0] = acc.sum; p[1] = acc.mx; p[2] = (double)acc.imx; p[3] = acc.mn; p[4] = (double)acc.imn;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    Acc tot{0.0, -INFINITY, INFINITY, 0x7fffffff, 0x7fffffff};
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kThreads) {
        const volatile double* p = scratch + 5 * k;
        merge(tot, Acc{p[0], p[1], p[3], (int)p[2], (int)p[4]});
    }
    tot = block_reduce(tot);
    if (threadIdx.x == 0) {
        result[0] = tot.sum / (double)n_face;
        result[1] = tot.mx; result[2] = (double)tot.imx;
        result[3] = tot.mn; result[4] = (double)tot.imn;
        *ticket = 0u;
    }
}

// Device address of g_scratch in the current context.  The runtime loads this library's module
// once per context, so the address is looked up (cudaGetSymbolAddress, with the device current)
// on the first call on each device and again whenever that device's current context is a
// different one: after cudaDeviceReset destroyed the primary context and a later call created a
// new one, the module is reloaded and the array may sit elsewhere.  Contexts are told apart by
// the driver's context ID, which is never reused within a process.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct ScratchSlot {
    unsigned long long ctx_id;
    double* addr;
};

std::mutex g_mu;
ScratchSlot g_slot[64] = {};
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// ID of the calling thread's current context, or false when there is none.
bool current_context_id(unsigned long long* id)
{
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
    return g_ctx_id(ctx, id) == CUDA_SUCCESS;
}

int scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_no_handle(LBM_ECUDA, "lbm_nusselt_static: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail_no_handle(LBM_ECUDA, "lbm_nusselt_static: device ordinal %d above 63", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ctx_current || !g_ctx_id) {
        void* p0 = nullptr;
        void* p1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
            q0 != cudaDriverEntryPointSuccess || !p0 ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &p1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || !p1)
            return fail_no_handle(LBM_ECUDA, "lbm_nusselt_static: cuCtxGetCurrent / cuCtxGetId are not available from the driver");
        g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(p0);
        g_ctx_id = reinterpret_cast<CtxGetIdFn>(p1);
    }
    unsigned long long id = 0;
    if (g_slot[dev].addr && current_context_id(&id) && id == g_slot[dev].ctx_id) {
        *out = g_slot[dev].addr;
        return LBM_OK;
    }
    // set-up: this also creates and makes current the device's primary context if needed
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return fail_no_handle(LBM_ECUDA, "lbm_nusselt_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    if (!current_context_id(&id)) return fail_no_handle(LBM_ECUDA, "lbm_nusselt_static: no current CUDA context");
    g_slot[dev] = ScratchSlot{id, static_cast<double*>(p)};
    *out = g_slot[dev].addr;
    return LBM_OK;
}
#undef err

}  // namespace
}  // namespace lbm

#define err(code, ...) lbm::fail_no_handle(code, "lbm_nusselt_static: " __VA_ARGS__)

extern "C" int lbm_nusselt_static(int lattice, int nx, int ny, int nz, const int face_kind[6],
                                  const double T_wall[6], double T_ref, const void* g, int face,
                                  double L, double dT, double* result, void* stream)
{
    using namespace lbm;
    const int lat = lattice & 0xff, pcode = lattice & ~0xff;
    if (lat != LBM_D2Q9_D2Q9 && lat != LBM_D3Q27_D3Q15) return err(LBM_EINVAL, "unknown lattice");
    const int dim = lat == LBM_D2Q9_D2Q9 ? 2 : 3;
    if (dim == 2 && nz == 0) nz = 1;
    if (nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1) || (long long)nx * ny * nz > INT_MAX)
        return err(LBM_EINVAL, "bad box dimensions %d x %d x %d", nx, ny, nz);
    if (!face_kind || !T_wall || !g || !result) return err(LBM_EINVAL, "NULL argument");
    if (face < 0 || face >= 2 * dim || face_kind[face] != LBM_WALL_FIXED_T)
        return err(LBM_EINVAL, "face %d is not a fixed-temperature wall of this box", face);
    if (!(L > 0) || !(dT > 0)) return err(LBM_EINVAL, "L and dT must be positive");
    const int ext[3] = {nx, ny, nz};
    if (ext[face / 2] < 2) return err(LBM_EINVAL, "fewer than two node layers normal to the face");
    const long long n_face = face / 2 == 0 ? (long long)ny * nz
                           : (face / 2 == 1 ? (long long)nx * nz : (long long)nx * ny);
    if (n_face > LBM_NUSSELT_STATIC_MAX_FACE_NODES)
        return err(LBM_EINVAL, "face %d has %lld nodes, more than LBM_NUSSELT_STATIC_MAX_FACE_NODES (%d), "
                   "the room of the fixed scratch array", face, n_face, (int)LBM_NUSSELT_STATIC_MAX_FACE_NODES);

    Geometry geo{};
    geo.nx = nx; geo.ny = ny; geo.nz = nz; geo.nxy = nx * ny; geo.n = nx * ny * nz;
    for (int f = 0; f < 6; ++f) {
        geo.kind[f] = (dim == 2 && f >= 4) ? LBM_PERIODIC : face_kind[f];
        if (geo.kind[f] < LBM_PERIODIC || geo.kind[f] > LBM_WALL_FIXED_T) return err(LBM_EINVAL, "bad face kind");
        geo.T_wall[f] = T_wall[f];
        geo.profile[f] = nullptr;
    }
    for (int ax = 0; ax < dim; ++ax)
        if ((geo.kind[2 * ax] == LBM_PERIODIC) != (geo.kind[2 * ax + 1] == LBM_PERIODIC))
            return err(LBM_EINVAL, "axis periodic on one face only");

    double* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != LBM_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the ticket must start at zero (a call interrupted earlier could have left it otherwise)
    cudaError_t e = cudaMemsetAsync(scratch + 5 * kMaxBlocks, 0, sizeof(double), st);
    if (e != cudaSuccess) return err(LBM_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    const double s = T_wall[face] >= T_ref ? 1.0 : -1.0;
    const double scale = -s * L / dT;
    const int blocks = (int)((n_face + kThreads - 1) / kThreads);
#define LBM_STATIC_LAUNCH(S, D)                                                               \
    nusselt_static_kernel<S, D><<<blocks, kThreads, 0, st>>>((const typename S::T*)g, geo, T_ref, \
                                                             face, (int)n_face, scale, scratch, result)
    if (pcode == LBM_FP64) {
        if (dim == 2) LBM_STATIC_LAUNCH(StoreF64, 2); else LBM_STATIC_LAUNCH(StoreF64, 3);
    } else if (pcode == LBM_FP32) {
        if (dim == 2) LBM_STATIC_LAUNCH(StoreF32, 2); else LBM_STATIC_LAUNCH(StoreF32, 3);
    } else if (pcode == LBM_FP16S) {
        if (dim == 2) LBM_STATIC_LAUNCH(StoreF16S, 2); else LBM_STATIC_LAUNCH(StoreF16S, 3);
    } else {
        return err(LBM_EINVAL, "unknown precision flag");
    }
#undef LBM_STATIC_LAUNCH
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(LBM_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return LBM_OK;
}
#undef err
