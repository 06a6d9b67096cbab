// batch.cu -- many independent 2D cavities (D2Q9 flow + D2Q9 energy) advanced by one kernel
// launch per time step.
//
// The members' populations are concatenated in two buffers (f and g, each with its own A/B copy);
// a device table holds every member's geometry, relaxation rates and buffer offset, and the
// first index of its tiles.  The launch has (SM count x CTAs per SM) blocks, usually more than
// the SMs hold at once, so the hardware block scheduler balances the shares (an oversubscribed
// grid, not a persistent one).  Block b takes an equal contiguous share of the global tile list,
// stages the owning member's table entry in shared memory (again only where its share crosses
// into the next member) and runs the same node step as the single-box kernel on one node per
// thread.  The
// tile shape and CTAs per SM come from lbm_batch_set_launch or from the autotuner
// lbm_batch_tune; the time loop replays CUDA graphs like lbm_step.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "kernels.h"
#include "step_d2q9.cuh"

namespace lbm {

template <class R>
struct BatchMember {
    Geometry geo;
    Coeffs2D<R> c;
    unsigned long long off;   // element offset of the member's planes in the f and g buffers
    int tile0;                // first global tile index of the member
    int tiles_x;              // tiles along x
};

// FP32 registers: at least 5 blocks of 256 threads (48 registers, no spills), i.e. 40 resident
// warps per SM for the memory pipeline; FP64 keeps the compiler's choice.
template <class S>
struct BatchBounds {
    static constexpr int kMinBlocks = sizeof(typename S::R) == 8 ? 1 : 5;
};

template <class S>
__global__ void __launch_bounds__(256, BatchBounds<S>::kMinBlocks)
    batch_step_d2q9_kernel(const typename S::T* __restrict__ fin, const typename S::T* __restrict__ gin,
                           typename S::T* __restrict__ fout, typename S::T* __restrict__ gout,
                           const BatchMember<typename S::R>* __restrict__ members, int n_members,
                           int n_tiles, int tile_x, int tile_y, unsigned* status)
{
    using M = BatchMember<typename S::R>;
    __shared__ __align__(16) unsigned char mbuf[sizeof(M)];
    const M& m = *reinterpret_cast<const M*>(mbuf);
    // block b owns the contiguous tile range [t0, t1): equal shares, the first `rem` blocks one more
    const int per = n_tiles / (int)gridDim.x, rem = n_tiles % (int)gridDim.x;
    const int t0 = (int)blockIdx.x * per + min((int)blockIdx.x, rem);
    const int t1 = t0 + per + ((int)blockIdx.x < rem ? 1 : 0);
    // owning member of t0 (every thread reads the same entries, so k is uniform in the block)
    int lo = 0, hi = n_members - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&members[mid].tile0) <= t0) lo = mid;
        else hi = mid - 1;
    }
    int k = lo, held = -1;
    for (int t = t0; t < t1; ++t) {
        while (k + 1 < n_members && __ldg(&members[k + 1].tile0) <= t) ++k;
        if (k != held) {
            __syncthreads();   // every thread is done with the previous member's entry
            const unsigned* src = reinterpret_cast<const unsigned*>(members + k);
            unsigned* dst = reinterpret_cast<unsigned*>(mbuf);
            for (int w = threadIdx.x; w < (int)(sizeof(M) / 4); w += blockDim.x) dst[w] = src[w];
            __syncthreads();
            held = k;
        }
        const int local = t - m.tile0;
        const int x = (local % m.tiles_x) * tile_x + (int)threadIdx.x % tile_x;
        const int y = (local / m.tiles_x) * tile_y + (int)threadIdx.x / tile_x;
        if (x < m.geo.nx && y < m.geo.ny)
            node_step_d2q9<S, unsigned>(fin + m.off, gin + m.off, fout + m.off, gout + m.off, m.geo, m.c,
                                        status + k, x, y);
    }
}

// Blocks of `threads` threads of the step kernel that fit on one SM at once.
template <class S>
static int resident_blocks(int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_d2q9_kernel<S>, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template <class S>
static cudaError_t launch_batch(const void* fin, const void* gin, void* fout, void* gout,
                                const void* members, int n_members, int n_tiles, int tile_x,
                                int tile_y, int grid, unsigned* status, cudaStream_t st)
{
    using T = typename S::T;
    batch_step_d2q9_kernel<S><<<grid, tile_x * tile_y, 0, st>>>(
        (const T*)fin, (const T*)gin, (T*)fout, (T*)gout,
        (const BatchMember<typename S::R>*)members, n_members, n_tiles, tile_x, tile_y, status);
    return cudaGetLastError();
}

}  // namespace lbm

struct lbm_batch_s {
    int prec = 0, count = 0;
    std::vector<lbm::BoxPlan> plans;
    std::vector<unsigned long long> off;
    std::vector<lbm_bc> bcs;
    unsigned long long total = 0;   // nodes of all members
    void* f[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    int cur = 0;
    void* members = nullptr;
    unsigned* status = nullptr;
    double *nu_profile = nullptr, *nu_scratch = nullptr, *nu_result = nullptr;
    unsigned* ticket = nullptr;
    int n_tiles = 0, tile_x = 64, tile_y = 2, ctas_per_sm = 0, sms = 0;
    cudaStream_t stream = nullptr, capture_stream = nullptr;
    int graph_steps = 32;
    unsigned gen = 1, graph_gen[2] = {0, 0};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long steps = 0;
    std::string err;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn dealloc = nullptr;
    void* actx = nullptr;
};

namespace {

thread_local std::string g_batch_create_error;

int bfail(lbm_batch_s* b, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    (b ? b->err : g_batch_create_error) = buf;
    return code;
}

#define B_CK(b, expr)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) return bfail(b, LBM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

void bfree(lbm_batch_s* b, void* p)
{
    if (p) b->dealloc(p, b->actx);
}

void brelease(lbm_batch_s* b)
{
    cudaStreamSynchronize(b->stream);
    for (int k = 0; k < 2; ++k) {
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
        bfree(b, b->f[k]);
        bfree(b, b->g[k]);
    }
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    bfree(b, b->members);
    bfree(b, b->status);
    bfree(b, b->nu_profile);
    bfree(b, b->nu_scratch);
    bfree(b, b->nu_result);
    bfree(b, b->ticket);
    delete b;
}

template <class R>
std::vector<lbm::BatchMember<R>> member_table(const lbm_batch_s* b)
{
    std::vector<lbm::BatchMember<R>> t(b->count);
    int tile = 0;
    for (int k = 0; k < b->count; ++k) {
        const lbm::BoxPlan& P = b->plans[k];
        t[k].geo = P.geo;
        t[k].c = lbm::make_coeffs<R, 9, 9>(P.hc);
        t[k].off = b->off[k];
        t[k].tile0 = tile;
        t[k].tiles_x = (P.nx + b->tile_x - 1) / b->tile_x;
        tile += t[k].tiles_x * ((P.ny + b->tile_y - 1) / b->tile_y);
    }
    return t;
}

// Upload the member table for the current tile shape.
int upload_table(lbm_batch_s* b)
{
    size_t bytes = 0;
    const void* src = nullptr;
    std::vector<lbm::BatchMember<double>> td;
    std::vector<lbm::BatchMember<float>> tf;
    if (b->prec == lbm::kF64) {
        td = member_table<double>(b);
        bytes = td.size() * sizeof(td[0]);
        src = td.data();
        b->n_tiles = td.back().tile0 + td.back().tiles_x * ((b->plans.back().ny + b->tile_y - 1) / b->tile_y);
    } else {
        tf = member_table<float>(b);
        bytes = tf.size() * sizeof(tf[0]);
        src = tf.data();
        b->n_tiles = tf.back().tile0 + tf.back().tiles_x * ((b->plans.back().ny + b->tile_y - 1) / b->tile_y);
    }
    if (!b->members) {
        const size_t cap = (size_t)b->count * std::max(sizeof(lbm::BatchMember<double>), sizeof(lbm::BatchMember<float>));
        b->members = b->alloc(cap, b->actx);
        if (!b->members) return bfail(b, LBM_ENOMEM, "no device memory for the member table");
    }
    B_CK(b, cudaMemcpyAsync(b->members, src, bytes, cudaMemcpyHostToDevice, b->stream));
    B_CK(b, cudaStreamSynchronize(b->stream));
    ++b->gen;
    return LBM_OK;
}

int max_resident(int prec, int threads);

// Blocks of one step launch: ctas_per_sm blocks per SM (0 = as many as are resident at once),
// at most one per tile.
int grid_of(lbm_batch_s* b)
{
    const int cps = b->ctas_per_sm > 0 ? b->ctas_per_sm : max_resident(b->prec, b->tile_x * b->tile_y);
    return std::max(1, std::min(b->n_tiles, b->sms * cps));
}

cudaError_t launch_one(lbm_batch_s* b, const void* fin, const void* gin, void* fout, void* gout,
                       cudaStream_t st)
{
    const int grid = grid_of(b);
    switch (b->prec) {
    case lbm::kF64: return lbm::launch_batch<lbm::StoreF64>(fin, gin, fout, gout, b->members, b->count, b->n_tiles, b->tile_x, b->tile_y, grid, b->status, st);
    case lbm::kF32: return lbm::launch_batch<lbm::StoreF32>(fin, gin, fout, gout, b->members, b->count, b->n_tiles, b->tile_x, b->tile_y, grid, b->status, st);
    case lbm::kF16S: return lbm::launch_batch<lbm::StoreF16S>(fin, gin, fout, gout, b->members, b->count, b->n_tiles, b->tile_x, b->tile_y, grid, b->status, st);
    }
    return cudaErrorInvalidValue;
}

int max_resident(int prec, int threads)
{
    switch (prec) {
    case lbm::kF64: return lbm::resident_blocks<lbm::StoreF64>(threads);
    case lbm::kF32: return lbm::resident_blocks<lbm::StoreF32>(threads);
    default: return lbm::resident_blocks<lbm::StoreF16S>(threads);
    }
}

int valid_launch(int tx, int ty, int cps)
{
    const int threads = tx * ty;
    return (tx == 32 || tx == 64 || tx == 128 || tx == 256) && ty >= 1 && threads <= 256 &&
           cps >= 0 && cps <= 1024;
}

size_t elem_bytes(int prec) { return lbm::storage_bytes(prec); }

int build_batch_graph(lbm_batch_s* b, int par)
{
    if (!b->capture_stream) B_CK(b, cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    if (b->graph[par]) {
        B_CK(b, cudaGraphExecDestroy(b->graph[par]));
        b->graph[par] = nullptr;
    }
    cudaGraph_t gr = nullptr;
    B_CK(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    int c = par;
    for (int t = 0; t < b->graph_steps && e == cudaSuccess; ++t) {
        e = launch_one(b, b->f[c], b->g[c], b->f[1 - c], b->g[1 - c], b->capture_stream);
        c = 1 - c;
    }
    const cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return bfail(b, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph[par], gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
    b->graph_gen[par] = b->gen;
    return LBM_OK;
}

int member_ok(lbm_batch_s* b, int member)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (member < 0 || member >= b->count) return bfail(b, LBM_EINVAL, "member %d out of range", member);
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(int lattice, int count, const int* nx, const int* ny, const double* Ra,
                     const double* Pr, double Ma, const lbm_bc* bc, lbm_batch* out)
{
    if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if ((lattice & 0xff) != LBM_D2Q9_D2Q9) return bfail(nullptr, LBM_ENOTSUP, "batches hold D2Q9 boxes");
    if (count < 1 || !nx || !ny || !Ra || !Pr || !bc) return bfail(nullptr, LBM_EINVAL, "empty batch or NULL array");
    lbm_batch_s* b = new lbm_batch_s;
    lbm::current_allocator(&b->alloc, &b->dealloc, &b->actx);
    b->count = count;
    b->plans.resize(count);
    b->off.resize(count);
    b->bcs.assign(bc, bc + count);
    for (int k = 0; k < count; ++k) {
        std::string e;
        const int rc = lbm::plan_box(lattice, nx[k], ny[k], 1, Ra[k], Pr[k], Ma, &bc[k], &b->plans[k], &e);
        if (rc) {
            delete b;
            return bfail(nullptr, rc, "member %d: %s", k, e.c_str());
        }
        if (!lbm::index32(b->plans[k].geo, 9)) {
            delete b;
            return bfail(nullptr, LBM_EINVAL, "member %d has more than 2^32 / 9 nodes", k);
        }
        b->off[k] = 9ULL * b->total;
        b->total += (unsigned long long)nx[k] * ny[k];
    }
    b->prec = b->plans[0].prec;
    // the global tile index is an int: at most total / 32 + count tiles for the narrowest tile
    if (b->total / 32 + (unsigned long long)count >= (unsigned long long)INT_MAX) {
        delete b;
        return bfail(nullptr, LBM_EINVAL, "batch of %llu nodes is too large", b->total);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->sms < 1) b->sms = 1;
    const size_t bytes = 9ULL * b->total * elem_bytes(b->prec);
    long max_face = 0;
    for (auto& P : b->plans) max_face = std::max<long>(max_face, std::max(P.nx, P.ny));
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) ok = (b->f[k] = b->alloc(bytes, b->actx)) && (b->g[k] = b->alloc(bytes, b->actx));
    ok = ok && (b->status = (unsigned*)b->alloc(sizeof(unsigned) * count, b->actx)) &&
         (b->nu_profile = (double*)b->alloc(sizeof(double) * max_face, b->actx)) &&
         (b->nu_scratch = (double*)b->alloc(sizeof(double) * lbm::nusselt_scratch_doubles(max_face), b->actx)) &&
         (b->nu_result = (double*)b->alloc(sizeof(double) * 8, b->actx)) &&
         (b->ticket = (unsigned*)b->alloc(sizeof(unsigned) * 4, b->actx));
    if (!ok) {
        bfail(nullptr, LBM_ENOMEM, "device allocation failed for a batch of %d members", count);
        brelease(b);
        return LBM_ENOMEM;
    }
    cudaError_t e = cudaMemsetAsync(b->status, 0, sizeof(unsigned) * count, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ticket, 0, sizeof(unsigned) * 4, b->stream);
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        const size_t o = b->off[k] * elem_bytes(b->prec);
        e = lbm::launch_init(2, b->prec, (char*)b->f[0] + o, (char*)b->g[0] + o, b->plans[k].geo,
                             bc[k].T_init, bc[k].T_ref, bc[k].seed, bc[k].perturb, b->stream);
    }
    if (e != cudaSuccess) {
        bfail(nullptr, LBM_ECUDA, "initialisation: %s", cudaGetErrorString(e));
        brelease(b);
        return LBM_ECUDA;
    }
    const int rc = upload_table(b);
    if (rc) {
        g_batch_create_error = b->err;
        brelease(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch b)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    brelease(b);
    return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch b, void* stream)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    b->stream = (cudaStream_t)stream;
    ++b->gen;
    return LBM_OK;
}

int lbm_batch_set_launch(lbm_batch b, int tile_x, int tile_y, int ctas_per_sm, int graph_steps)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (!valid_launch(tile_x, tile_y, ctas_per_sm))
        return bfail(b, LBM_EINVAL, "tile %d x %d with %d CTAs per SM is not a valid launch", tile_x, tile_y, ctas_per_sm);
    if (graph_steps < 0 || graph_steps > 4096) return bfail(b, LBM_EINVAL, "graph_steps must be in [0, 4096]");
    b->tile_x = tile_x;
    b->tile_y = tile_y;
    b->ctas_per_sm = ctas_per_sm;
    b->graph_steps = graph_steps + (graph_steps & 1);
    return upload_table(b);
}

int lbm_batch_step(lbm_batch b, long n)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (n < 0) return bfail(b, LBM_EINVAL, "negative step count");
    const lbm::NvtxRange range("lbm_batch_step");
    while (b->graph_steps > 0 && n >= b->graph_steps) {
        const int par = b->cur;
        if (!b->graph[par] || b->graph_gen[par] != b->gen) {
            const int rc = build_batch_graph(b, par);
            if (rc) return rc;
        }
        B_CK(b, cudaGraphLaunch(b->graph[par], b->stream));
        b->steps += b->graph_steps;
        n -= b->graph_steps;
    }
    for (long t = 0; t < n; ++t) {
        const int c = b->cur;
        B_CK(b, launch_one(b, b->f[c], b->g[c], b->f[1 - c], b->g[1 - c], b->stream));
        b->cur = 1 - c;
        ++b->steps;
    }
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch b, int trial_steps, int* tile_x, int* tile_y, int* ctas_per_sm)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (trial_steps < 1) return bfail(b, LBM_EINVAL, "trial_steps must be positive");
    // keep the state: the trials advance a copy of the populations, not the batch
    const size_t bytes = 9ULL * b->total * elem_bytes(b->prec);
    void* tf[2] = {b->alloc(bytes, b->actx), b->alloc(bytes, b->actx)};
    void* tg[2] = {b->alloc(bytes, b->actx), b->alloc(bytes, b->actx)};
    if (!tf[0] || !tf[1] || !tg[0] || !tg[1]) {
        for (void* p : {tf[0], tf[1], tg[0], tg[1]}) bfree(b, p);
        return bfail(b, LBM_ENOMEM, "no device memory for the tuning copy");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // each tile shape with 1/2 to 64 times the blocks that are resident on an SM at once (at most
    // 1024): oversubscribed grids let the block scheduler even out the uneven members
    const int shapes[][2] = {{32, 2}, {32, 4}, {64, 1}, {64, 2}, {64, 4}, {128, 1}, {128, 2}, {256, 1}};
    const int keep[3] = {b->tile_x, b->tile_y, b->ctas_per_sm};
    float best = INFINITY;
    int bx = keep[0], by = keep[1], bc = keep[2];
    int rc = LBM_OK;
    cudaMemcpyAsync(tf[0], b->f[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(tg[0], b->g[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream);
    for (auto& sh : shapes) {
        const int occ = max_resident(b->prec, sh[0] * sh[1]);
        const int ctas[8] = {std::max(1, occ / 2), occ, 2 * occ, 4 * occ, 8 * occ, 16 * occ, 32 * occ, 64 * occ};
        int last = 0;
        for (int cps : ctas) {
            cps = std::min(cps, 1024);
            if (cps == last || !valid_launch(sh[0], sh[1], cps)) continue;
            last = cps;
            b->tile_x = sh[0];
            b->tile_y = sh[1];
            b->ctas_per_sm = cps;
            if ((rc = upload_table(b))) break;
            int c = 0;
            for (int t = 0; t < 2 + trial_steps; ++t) {
                if (t == 2) cudaEventRecord(e0, b->stream);
                launch_one(b, tf[c], tg[c], tf[1 - c], tg[1 - c], b->stream);
                c = 1 - c;
            }
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (cudaGetLastError() == cudaSuccess && ms < best) {
                best = ms;
                bx = sh[0];
                by = sh[1];
                bc = cps;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(b->stream);
    for (void* p : {tf[0], tf[1], tg[0], tg[1]}) bfree(b, p);
    // the trial steps may have flagged members that the real state has not: clear, then re-check
    cudaMemsetAsync(b->status, 0, sizeof(unsigned) * b->count, b->stream);
    b->tile_x = bx;
    b->tile_y = by;
    b->ctas_per_sm = bc;
    if (!rc) rc = upload_table(b);
    if (tile_x) *tile_x = bx;
    if (tile_y) *tile_y = by;
    if (ctas_per_sm) *ctas_per_sm = bc;
    return rc;
}

int lbm_batch_sync(lbm_batch b, int* diverged)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    std::vector<unsigned> st(b->count);
    B_CK(b, cudaMemcpyAsync(st.data(), b->status, sizeof(unsigned) * b->count, cudaMemcpyDeviceToHost, b->stream));
    B_CK(b, cudaStreamSynchronize(b->stream));
    int nbad = 0;
    for (int k = 0; k < b->count; ++k) {
        if (diverged) diverged[k] = st[k] ? 1 : 0;
        nbad += st[k] ? 1 : 0;
    }
    if (nbad) return bfail(b, LBM_EDIVERGED, "%d of %d members diverged", nbad, b->count);
    return LBM_OK;
}

int lbm_batch_nusselt(lbm_batch b, int member, int face, double* mean, double* nu_max,
                      double* nu_min, int* j_max, int* j_min)
{
    int rc = member_ok(b, member);
    if (rc) return rc;
    const lbm::BoxPlan& P = b->plans[member];
    if (face < 0 || face >= 4 || P.geo.kind[face] != LBM_WALL_FIXED_T)
        return bfail(b, LBM_EINVAL, "face %d is not a fixed-temperature wall of member %d", face, member);
    const int ext[2] = {P.nx, P.ny};
    if (ext[face / 2] < 2) return bfail(b, LBM_EINVAL, "fewer than two node layers normal to face %d", face);
    const double s = P.geo.T_wall[face] >= P.hc.T_ref ? 1.0 : -1.0;
    const size_t o = b->off[member] * elem_bytes(b->prec);
    B_CK(b, lbm::launch_nusselt(2, b->prec, (char*)b->f[b->cur] + o, (char*)b->g[b->cur] + o, P.geo, P.hc,
                                face, -s * P.L / P.dT, b->nu_profile, b->nu_scratch, b->ticket,
                                b->nu_result, b->stream));
    double r[5];
    B_CK(b, cudaMemcpyAsync(r, b->nu_result, sizeof r, cudaMemcpyDeviceToHost, b->stream));
    B_CK(b, cudaStreamSynchronize(b->stream));
    const long n = face < 2 ? P.ny : P.nx;
    if (mean) *mean = r[0] / (double)n;
    if (nu_max) *nu_max = r[1];
    if (j_max) *j_max = (int)r[2];
    if (nu_min) *nu_min = r[3];
    if (j_min) *j_min = (int)r[4];
    return LBM_OK;
}

int lbm_batch_get_populations(lbm_batch b, int member, double* f, double* g)
{
    int rc = member_ok(b, member);
    if (rc) return rc;
    if (!f || !g) return bfail(b, LBM_EINVAL, "NULL output");
    const lbm::BoxPlan& P = b->plans[member];
    const size_t n = (size_t)P.geo.n, o = b->off[member] * elem_bytes(b->prec);
    double* tmp = (double*)b->alloc(18 * n * sizeof(double), b->actx);
    if (!tmp) return bfail(b, LBM_ENOMEM, "no device memory for the staging buffer");
    cudaError_t e = lbm::launch_get_pops(2, b->prec, (char*)b->f[b->cur] + o, (char*)b->g[b->cur] + o, P.geo,
                                         P.hc.T_ref, tmp, tmp + 9 * n, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, tmp, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g, tmp + 9 * n, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaStreamSynchronize(b->stream);
    bfree(b, tmp);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "%s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_batch_set_populations(lbm_batch b, int member, const double* f, const double* g)
{
    int rc = member_ok(b, member);
    if (rc) return rc;
    if (!f || !g) return bfail(b, LBM_EINVAL, "NULL input");
    const lbm::BoxPlan& P = b->plans[member];
    const size_t n = (size_t)P.geo.n, o = b->off[member] * elem_bytes(b->prec);
    double* tmp = (double*)b->alloc(18 * n * sizeof(double), b->actx);
    if (!tmp) return bfail(b, LBM_ENOMEM, "no device memory for the staging buffer");
    cudaError_t e = cudaMemcpyAsync(tmp, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp + 9 * n, g, 9 * n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = lbm::launch_set_pops(2, b->prec, (char*)b->f[b->cur] + o, (char*)b->g[b->cur] + o, P.geo, P.hc.T_ref,
                                 tmp, tmp + 9 * n, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaStreamSynchronize(b->stream);
    bfree(b, tmp);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "%s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_batch_info(lbm_batch b, lbm_batch_info_t* o)
{
    if (!b || !o) return bfail(b, LBM_EINVAL, "batch or output is NULL");
    o->count = b->count;
    o->total_nodes = (long long)b->total;
    o->n_tiles = b->n_tiles;
    o->tile_x = b->tile_x;
    o->tile_y = b->tile_y;
    o->ctas_per_sm = b->ctas_per_sm > 0 ? b->ctas_per_sm : max_resident(b->prec, b->tile_x * b->tile_y);
    o->grid = grid_of(b);
    o->graph_steps = b->graph_steps;
    o->steps = b->steps;
    o->bytes_per_node_update = 2.0 * 18 * (double)elem_bytes(b->prec);
    return LBM_OK;
}

const char* lbm_batch_last_error(lbm_batch b)
{
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

}  // extern "C"
