// step_d3q27_tma.cuh -- the fused D3Q27 + D3Q15 step with its pull staged through shared memory
// by the tensor memory accelerator (TMA).
//
// A persistent grid walks tiles of 64 x TY nodes of one z-plane.  For every tile, a producer
// thread issues 42 tensor loads, one per population plane a: the box of the nodes that the
// tile's links along e_a pull from, starting at (x0 - H, y0 - e_ay, z0 - e_az), where H is
// 16 bytes of elements (4 in FP32, 8 in FP16).  Starting H nodes left of the tile keeps the box's
// x coordinate on a 16-byte boundary, as a tensor copy requires; a node then finds its upwind
// value at column lx + H - e_ax of that 64 + 2H wide box.  The boxes land in a ring of stages;
// while the consumer warps collide one tile, the copies of the next ones are in flight.
//
// Boundaries: tiles that touch a y or z wall or wrap take the global-memory pull of the plain
// kernel.  In the other tiles, the nodes on an x wall (or x wrap) replace only their links that
// leave through x, with the wall rules read from global memory.  Boxes are zero-filled outside
// the box, and those values are never used.
//
// Waits on the mbarriers are bounded: after about a second the block records bit 1 in the status
// word, stops, and waits (again bounded) for its copies still in flight before it returns.
#pragma once

#include <cuda.h>

#include "step_d3q27.cuh"

namespace lbm {

constexpr int kTmaTX = 64;   // tile width (nodes along x) = threads along x

// Shared-memory slab of one population: TY rows of kBoxX elements, padded to 128 bytes.
template <class T, int TY>
struct TmaLayout {
    static constexpr int kHalo = 16 / (int)sizeof(T);        // 16 bytes of nodes on each side
    static constexpr int kBoxX = kTmaTX + 2 * kHalo;          // box width (a multiple of 16 bytes)
    static constexpr int kSlabBytes = ((TY * kBoxX * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int kSlabElems = kSlabBytes / (int)sizeof(T);
    static constexpr int kStageBytes = 42 * kSlabBytes;
    static constexpr int kStages = 3;
    static constexpr int kSmemBytes = kStages * kStageBytes + 128;   // the ring + its mbarriers
    static constexpr unsigned kTileBytes = 42u * TY * kBoxX * sizeof(T);   // bytes landed per tile
    // blocks that fit in one SM's 228 KB of shared memory (1 KB of it reserved per block)
    static constexpr int kMinBlocks = (228 * 1024) / (kSmemBytes + 1024) > 0 ? (228 * 1024) / (kSmemBytes + 1024) : 1;
};

__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Spin until the phase with this parity has completed, for at most ~limit clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// 4D tensor load (x, y, z, plane) into shared memory, completing on the mbarrier.
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Order this thread's earlier generic-proxy accesses to shared memory before later async-proxy
// (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Value of a stored element as a deviation from its rest value (storage policy S).
template <class S>
__device__ __forceinline__ typename S::R dev_of(typename S::T v, typename S::R shift);
template <>
__device__ __forceinline__ double dev_of<StoreF64>(double v, double shift) { return v - shift; }
template <>
__device__ __forceinline__ float dev_of<StoreF32>(float v, float) { return v; }
template <>
__device__ __forceinline__ float dev_of<StoreF16S>(__half v, float)
{
    return __half2float(v) * StoreF16S::kInvScale;
}

template <class S, int TY>
__device__ __forceinline__ void tma_issue_tile(const CUtensorMap* mf, const CUtensorMap* mg,
                                               unsigned stage, unsigned bar, int x0, int y0, int z)
{
    using L = TmaLayout<typename S::T, TY>;
    mbar_arrive_expect_tx(bar, L::kTileBytes);
    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        tma_load_4d(stage + a * L::kSlabBytes, mf, x0 - L::kHalo, y0 - e27(a, 1), z - e27(a, 2), a, bar);
    });
    static_for<15>([&](auto B) {
        constexpr int b = decltype(B)::value;
        tma_load_4d(stage + (27 + b) * L::kSlabBytes, mg, x0 - L::kHalo, y0 - e15(b, 1), z - e15(b, 2), b, bar);
    });
}

// Links of a node on an x wall (or x wrap) that leave the box through x, replaced by the wall
// rules (or the wrapped source) from global memory; the other links keep their staged values.
template <class S, class Idx>
__device__ __forceinline__ void fix_x_edge_d3q27(const typename S::T* __restrict__ fin,
                                                 const typename S::T* __restrict__ gin,
                                                 const Geometry& geo, int x, int y, int z, int i,
                                                 typename S::R T_ref, typename S::R f[27],
                                                 typename S::R g[15])
{
    using R = typename S::R;
    const NodeWalls<R> w = node_walls_x<R>(geo, x, y, z);
    static_for<27>([&](auto A) {
        constexpr int a = decltype(A)::value;
        constexpr int ex = e27(a, 0);
        if constexpr (ex != 0) {
            const bool leaves = ex == 1 ? x == 0 : x == geo.nx - 1;
            if (leaves) {
                constexpr int o = opp27(a);
                bool out, dir;
                R tw;
                const int s = link_source<ex, e27(a, 1), e27(a, 2)>(geo, w, i, &out, &dir, &tw);
                const Idx off = out ? (Idx)o * geo.n + i : (Idx)a * geo.n + s;
                f[a] = S::load_dev(fin, off, R(w27(a)));
                constexpr int b = g15_of_27(a);
                if constexpr (b >= 0) {
                    constexpr int ob = opp15(b);
                    const Idx og = out ? (Idx)ob * geo.n + i : (Idx)b * geo.n + s;
                    const R gv = S::load_dev(gin, og, R(w15(b)) * T_ref);
                    g[b] = dir ? R(2.0 * w15(b)) * (tw - T_ref) - gv : gv;
                }
            }
        }
    });
}

// Block: TY rows of 64 consumer threads (one node each) and one producer warp whose first lane
// issues the tensor copies.  The tiles of a block are a contiguous range of the tile list (x
// fastest, then y, then z), walked with incrementally updated coordinates.  Stage s of the
// kStages-deep ring has a "full" barrier (the copies of its tile have landed) and an "empty"
// barrier (every consumer warp is done with it); no block-wide barrier is used in the loop.
template <class S, class Idx, int TY, int kRates = 0>
__global__ void __launch_bounds__(kTmaTX * TY + 32, TmaLayout<typename S::T, TY>::kMinBlocks)
    step_d3q27_tma_kernel(const __grid_constant__ CUtensorMap mf, const __grid_constant__ CUtensorMap mg,
                          const typename S::T* __restrict__ fin, const typename S::T* __restrict__ gin,
                          typename S::T* __restrict__ fout, typename S::T* __restrict__ gout,
                          Geometry geo, Coeffs3D<typename S::R> c, unsigned* status, int tiles_x,
                          int tiles_y, int n_tiles)
{
    using R = typename S::R;
    using T = typename S::T;
    using L = TmaLayout<T, TY>;
    constexpr int NS = L::kStages;
    constexpr int NC = kTmaTX * TY;          // consumer threads
    constexpr int NCW = NC / 32;             // consumer warps
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + NS * L::kStageBytes);
    const unsigned smem0 = smem_addr(smem);
    auto full_bar = [&](int st) { return smem_addr(bars + st); };
    auto empty_bar = [&](int st) { return smem_addr(bars + NS + st); };
    const int tid = threadIdx.x, lane = tid & 31;
    const long long kWaitLimit = 2000000000LL;   // ~1 s at 2 GHz

    if (tid == 0) {
        for (int st = 0; st < NS; ++st) {
            mbar_init(full_bar(st), 1);
            mbar_init(empty_bar(st), NCW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    // contiguous share of the tiles: equal parts, the first `rem` blocks one more
    const int per = n_tiles / (int)gridDim.x, rem = n_tiles % (int)gridDim.x;
    const int t0 = (int)blockIdx.x * per + min((int)blockIdx.x, rem);
    const int t1 = t0 + per + ((int)blockIdx.x < rem ? 1 : 0);
    int tx = t0 % tiles_x, ty = (t0 / tiles_x) % tiles_y, tz = t0 / tiles_x / tiles_y;
    // tensor copies need a 128-byte aligned destination; otherwise every tile pulls from global
    const bool smem_ok = (smem0 & 127u) == 0;
    auto staged_tile = [&](int y0, int z) {
        return smem_ok && y0 >= 1 && y0 + TY <= geo.ny - 1 && z >= 1 && z <= geo.nz - 2;
    };
    auto advance = [&]() {
        if (++tx == tiles_x) {
            tx = 0;
            if (++ty == tiles_y) {
                ty = 0;
                ++tz;
            }
        }
    };

    bool failed = false;
    int issued = 0;
    if (tid >= NC) {
        // producer warp: lane 0 keeps the ring full
        if (lane == 0) {
            for (int t = t0; t < t1; ++t, ++issued, advance()) {
                const int st = issued % NS, round = issued / NS;
                if (round > 0 && !mbar_wait_bounded(empty_bar(st), (round - 1) & 1, kWaitLimit)) {
                    failed = true;
                    break;
                }
                const int x0 = tx * kTmaTX, y0 = ty * TY;
                if (staged_tile(y0, tz)) {
                    fence_proxy_async_smem();
                    tma_issue_tile<S, TY>(&mf, &mg, smem0 + st * L::kStageBytes, full_bar(st), x0, y0, tz);
                } else {
                    mbar_arrive(full_bar(st));   // nothing to stage: complete the phase at once
                }
            }
        }
    } else {
        const int lx = tid % kTmaTX, ly = tid / kTmaTX;
        for (int t = t0, k = 0; t < t1; ++t, ++k, advance()) {
            const int st = k % NS, round = k / NS;
            const bool ok = mbar_wait_bounded(full_bar(st), round & 1, kWaitLimit);
            if (!__all_sync(0xffffffffu, ok)) {
                failed = true;
                break;
            }
            const int x0 = tx * kTmaTX, y0 = ty * TY;
            const int x = x0 + lx, y = y0 + ly, z = tz;
            if (x < geo.nx && y < geo.ny) {
                const int i = x + geo.nx * y + geo.nxy * z;
                R f[27], g[15];
                if (staged_tile(y0, z)) {
                    const T* sb = reinterpret_cast<const T*>(smem + st * L::kStageBytes) + ly * L::kBoxX + lx + L::kHalo;
                    static_for<27>([&](auto A) {
                        constexpr int a = decltype(A)::value;
                        f[a] = dev_of<S>(sb[a * L::kSlabElems - e27(a, 0)], R(w27(a)));
                    });
                    static_for<15>([&](auto B) {
                        constexpr int b = decltype(B)::value;
                        g[b] = dev_of<S>(sb[(27 + b) * L::kSlabElems - e15(b, 0)], R(w15(b)) * c.T_ref);
                    });
                    if (x == 0 || x == geo.nx - 1)
                        fix_x_edge_d3q27<S, Idx>(fin, gin, geo, x, y, z, i, c.T_ref, f, g);
                } else if (x > 0 && x < geo.nx - 1 && y > 0 && y < geo.ny - 1 && z > 0 && z < geo.nz - 1) {
                    pull_d3q27_d3q15_interior<S, Idx>(fin, gin, geo, i, c.T_ref, f, g);
                } else {
                    const NodeWalls<R> w = node_walls<R>(geo, x, y, z, 3);
                    pull_d3q27_d3q15<S, Idx>(fin, gin, geo, w, i, c.T_ref, f, g);
                }
                collide_store_d3q27<S, Idx, kRates>(f, g, fout, gout, geo, c, status, i);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_bar(st));   // this warp is done with stage st
        }
    }
    if (__syncthreads_or(failed)) {
        if (tid == NC) {
            atomicOr(status, 2u);
            // copies still in flight write into this block's shared memory: wait for the last
            // phases the producer issued, again with a limit
            for (int j = max(0, issued - NS); j < issued; ++j)
                mbar_wait_bounded(full_bar(j % NS), (j / NS) & 1, kWaitLimit);
        }
        __syncthreads();
    }
}

}  // namespace lbm
