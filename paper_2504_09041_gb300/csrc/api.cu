// api.cu -- the C ABI of liblbm.so (declared in include/lbm.h).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "kernels.h"

namespace {

void* default_alloc(size_t bytes, void*)
{
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void default_free(void* p, void*) { cudaFree(p); }

lbm_alloc_fn g_alloc = default_alloc;
lbm_free_fn g_free = default_free;
void* g_ctx = nullptr;
thread_local std::string g_create_error;

constexpr unsigned long long kStateMagic = 0x46504c424d535431ULL;  // "FPLBMST1"
constexpr size_t kStateHeader = 64;

}  // namespace

struct lbm_s {
    int lattice = 0, prec = 0, dim = 0, nx = 0, ny = 0, nz = 0, qf = 0, qg = 0;
    lbm::Geometry geo{};
    lbm::HostCoeffs hc{};
    lbm_bc bc{};
    double L = 0, dT = 1, U = 0, nu = 0, alpha = 0;
    void* f[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    int cur = 0;
    double* profile[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double* nu_profile = nullptr;   // max face nodes
    double* nu_scratch = nullptr;   // block partials
    double* nu_result = nullptr;    // 5 doubles
    unsigned* ticket = nullptr;
    unsigned* status = nullptr;
    cudaStream_t stream = nullptr;
    int block_x = 0, block_y = 0;   // launch shape of the step kernel (0: default)
    int adjoint_arith = 2;          // arithmetic of the adjoint's VJPs: 0 FP32, 1 FP64, 2 double-float
    int adjoint_overlap = 1;        // recompute the next segment on a second stream beside the adjoint steps
    int tma_rows = 0;               // 3D FP32/FP16S: TMA-staged step with tiles of 64 x tma_rows
    lbm::TmaMaps tm[2];             // tensor maps of the input buffers f[c], g[c]
    // CUDA graphs of graph_steps consecutive steps (even, so the A/B parity returns), one per
    // starting parity, rebuilt whenever a launch parameter changes (gen != graph_gen)
    int graph_steps = 32;
    unsigned gen = 1, graph_gen[2] = {0, 0};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaStream_t capture_stream = nullptr;
    cudaStream_t aux_stream = nullptr;   // adjoint: recompute of the next segment, beside the adjoint steps
    long long steps = 0;
    std::string err;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn dealloc = nullptr;
    void* actx = nullptr;
};

namespace {

int fail(lbm_s* h, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return code;
}

#define LBM_CK(h, expr)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) return fail(h, LBM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

void* dev_alloc(lbm_s* h, size_t bytes)
{
    return h->alloc(bytes, h->actx);
}
void dev_free(lbm_s* h, void* p)
{
    if (p) h->dealloc(p, h->actx);
}

void release(lbm_s* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (int k = 0; k < 2; ++k)
        if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->aux_stream) {
        cudaStreamSynchronize(h->aux_stream);
        cudaStreamDestroy(h->aux_stream);
    }
    for (int k = 0; k < 2; ++k) {
        dev_free(h, h->f[k]);
        dev_free(h, h->g[k]);
    }
    for (int k = 0; k < 6; ++k) dev_free(h, h->profile[k]);
    dev_free(h, h->nu_profile);
    dev_free(h, h->nu_scratch);
    dev_free(h, h->nu_result);
    dev_free(h, h->ticket);
    dev_free(h, h->status);
    delete h;
}

bool rate_ok(double w) { return std::isfinite(w) && w > 0.0 && w < 2.0; }

long face_nodes(const lbm_s* h, int face)
{
    const int ax = face / 2;
    if (ax == 0) return (long)h->ny * h->nz;
    if (ax == 1) return (long)h->nx * h->nz;
    return (long)h->nx * h->ny;
}

size_t pop_bytes(const lbm_s* h)
{
    return (size_t)(h->qf + h->qg) * (size_t)h->geo.n * lbm::storage_bytes(h->prec);
}

// Device temporary of n doubles for host <-> device staging.
struct Tmp {
    lbm_s* h;
    double* p = nullptr;
    Tmp(lbm_s* hh, size_t n) : h(hh) { p = (double*)dev_alloc(h, n * sizeof(double)); }
    ~Tmp()
    {
        if (p) {
            cudaStreamSynchronize(h->stream);
            dev_free(h, p);
        }
    }
};

}  // namespace

extern "C" {

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void* ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(nullptr, LBM_EINVAL, "allocator: give both functions or neither");
    g_alloc = alloc ? alloc : default_alloc;
    g_free = free_fn ? free_fn : default_free;
    g_ctx = alloc ? ctx : nullptr;
    return LBM_OK;
}

const char* lbm_status_string(int s)
{
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of device memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EDIVERGED: return "simulation diverged";
    case LBM_ETIMEOUT: return "a bounded device wait timed out";
    case LBM_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

const char* lbm_last_error(lbm_handle h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

namespace lbm {

int fail_no_handle(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_create_error = buf;
    return code;
}

void current_allocator(lbm_alloc_fn* a, lbm_free_fn* f, void** ctx)
{
    *a = g_alloc;
    *f = g_free;
    *ctx = g_ctx;
}

// Validate a box description and derive its parameters (Sec. 6.1, Sec. 7): L across the fixed-T
// faces, U = Ma / sqrt(3), g beta dT L = U^2, nu = U L sqrt(Pr / Ra), alpha = nu / Pr, and the
// rates of App. A/B/C.  On failure returns the status and sets *err.
int plan_box(int lattice, int nx, int ny, int nz, double Ra, double Pr, double Ma, const lbm_bc* bc,
             BoxPlan* P, std::string* err)
{
    char buf[256];
    auto bad = [&](int code, const char* fmt, auto... a) {
        snprintf(buf, sizeof buf, fmt, a...);
        *err = buf;
        return code;
    };
    const int lat = lattice & 0xff;
    const int prec_code = lattice & ~0xff;
    if (lat != LBM_D2Q9_D2Q9 && lat != LBM_D3Q27_D3Q15) return bad(LBM_EINVAL, "unknown lattice %d", lat);
    int prec;
    if (prec_code == LBM_FP64) prec = kF64;
    else if (prec_code == LBM_FP32) prec = kF32;
    else if (prec_code == LBM_FP16S) prec = kF16S;
    else return bad(LBM_EINVAL, "unknown precision flag 0x%x", prec_code);
    const int dim = lat == LBM_D2Q9_D2Q9 ? 2 : 3;
    if (dim == 2 && nz == 0) nz = 1;
    if (nx < 1 || ny < 1 || nz < 1) return bad(LBM_EINVAL, "box %d x %d x %d is empty", nx, ny, nz);
    if (dim == 2 && nz != 1) return bad(LBM_EINVAL, "2D boxes need nz = 1");
    if ((long long)nx * ny * nz > INT_MAX) return bad(LBM_EINVAL, "more than 2^31 - 1 nodes");
    if (nz > 65535 || (ny + 1) / 2 > 65535) return bad(LBM_EINVAL, "box too tall for the launch grid");
    if (!(std::isfinite(Ra) && Ra > 0) || !(std::isfinite(Pr) && Pr > 0) || !(std::isfinite(Ma) && Ma > 0))
        return bad(LBM_EINVAL, "Ra, Pr and Ma must be positive and finite");
    if (!bc) return bad(LBM_EINVAL, "bc is NULL");
    for (int f = 0; f < 6; ++f)
        if (bc->face[f] < LBM_PERIODIC || bc->face[f] > LBM_WALL_FIXED_T)
            return bad(LBM_EINVAL, "face %d: unknown kind %d", f, bc->face[f]);
    for (int ax = 0; ax < dim; ++ax)
        if ((bc->face[2 * ax] == LBM_PERIODIC) != (bc->face[2 * ax + 1] == LBM_PERIODIC))
            return bad(LBM_EINVAL, "axis %d is periodic on one face only", ax);
    if (bc->gravity_axis < 0 || bc->gravity_axis >= dim)
        return bad(LBM_EINVAL, "gravity axis %d out of range", bc->gravity_axis);

    P->lattice = lat;
    P->prec = prec;
    P->dim = dim;
    P->nx = nx;
    P->ny = ny;
    P->nz = nz;
    P->qf = dim == 2 ? 9 : 27;
    P->qg = dim == 2 ? 9 : 15;
    Geometry& g = P->geo;
    g = Geometry{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.nxy = nx * ny;
    g.n = nx * ny * nz;
    for (int f = 0; f < 6; ++f) {
        g.kind[f] = (dim == 2 && f >= 4) ? LBM_PERIODIC : bc->face[f];
        g.T_wall[f] = bc->T_wall[f];
        g.profile[f] = nullptr;
    }
    const int ext[3] = {nx, ny, nz};
    P->L = nx;
    double tmin = INFINITY, tmax = -INFINITY;
    int nfixed = 0;
    for (int f = 2 * dim - 1; f >= 0; --f)
        if (g.kind[f] == LBM_WALL_FIXED_T) P->L = ext[f / 2];
    for (int f = 0; f < 2 * dim; ++f)
        if (g.kind[f] == LBM_WALL_FIXED_T) {
            ++nfixed;
            tmin = fmin(tmin, bc->T_wall[f]);
            tmax = fmax(tmax, bc->T_wall[f]);
        }
    P->dT = (nfixed >= 2 && tmax > tmin) ? tmax - tmin : 1.0;
    P->U = Ma / std::sqrt(3.0);
    P->nu = P->U * P->L * std::sqrt(Pr / Ra);
    P->alpha = P->nu / Pr;
    HostCoeffs& hc = P->hc;
    hc = HostCoeffs{};
    hc.gbeta = P->U * P->U / (P->L * P->dT);
    hc.T_ref = bc->T_ref;
    hc.gaxis = bc->gravity_axis;
    hc.fp16_sr = 1;
    hc.adj_sync = 2;   // adjoint step: 128 x 2 blocks with phase barriers (measured fastest)
    hc.rows3d = 0;     // 3D FP32 / FP16S step: rows per thread chosen per form (rows3d_for)
    const double om_nu = 1.0 / (3.0 * P->nu + 0.5);
    const double om_alpha = 1.0 / (3.0 * P->alpha + 0.5);
    // App. A, B, C: shear / diffusivity rates from nu / alpha, bulk and every free rate 1
    for (int a = 0; a < 27; ++a) hc.om_f[a] = 1.0;
    for (int b = 0; b < 15; ++b) hc.om_g[b] = 1.0;
    if (dim == 2) {
        hc.om_f[4] = hc.om_f[5] = om_nu;
        hc.om_g[1] = hc.om_g[2] = om_alpha;
    } else {
        hc.om_f[4] = hc.om_f[5] = hc.om_f[6] = om_nu;
        hc.om_f[8] = hc.om_f[9] = om_nu;
        hc.om_g[1] = hc.om_g[2] = hc.om_g[3] = om_alpha;
    }
    return LBM_OK;
}

}  // namespace lbm

extern "C" {

int lbm_create(int lattice, int nx, int ny, int nz, double Ra, double Pr, double Ma,
               const lbm_bc* bc, lbm_handle* out)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm::BoxPlan P;
    std::string err;
    const int rc = lbm::plan_box(lattice, nx, ny, nz, Ra, Pr, Ma, bc, &P, &err);
    if (rc) return fail(nullptr, rc, "%s", err.c_str());
    const int prec = P.prec, dim = P.dim;
    nx = P.nx;
    ny = P.ny;
    nz = P.nz;

    lbm_s* h = new lbm_s;
    h->alloc = g_alloc;
    h->dealloc = g_free;
    h->actx = g_ctx;
    h->lattice = P.lattice;
    h->prec = prec;
    h->dim = dim;
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->qf = P.qf;
    h->qg = P.qg;
    h->bc = *bc;
    h->geo = P.geo;
    lbm::Geometry& g = h->geo;
    h->L = P.L;
    h->dT = P.dT;
    h->U = P.U;
    h->nu = P.nu;
    h->alpha = P.alpha;
    h->hc = P.hc;

    // Device memory.
    const size_t sb = lbm::storage_bytes(prec);
    long max_face = 0;
    for (int f = 0; f < 2 * dim; ++f) max_face = std::max(max_face, face_nodes(h, f));
    for (int k = 0; k < 2; ++k) {
        h->f[k] = dev_alloc(h, (size_t)h->qf * g.n * sb);
        h->g[k] = dev_alloc(h, (size_t)h->qg * g.n * sb);
    }
    h->nu_profile = (double*)dev_alloc(h, sizeof(double) * max_face);
    h->nu_scratch = (double*)dev_alloc(h, sizeof(double) * lbm::nusselt_scratch_doubles(max_face));
    h->nu_result = (double*)dev_alloc(h, sizeof(double) * 8);
    h->ticket = (unsigned*)dev_alloc(h, sizeof(unsigned) * 4);
    h->status = (unsigned*)dev_alloc(h, sizeof(unsigned) * 4);
    if (!h->f[0] || !h->f[1] || !h->g[0] || !h->g[1] || !h->nu_profile || !h->nu_scratch ||
        !h->nu_result || !h->ticket || !h->status) {
        fail(nullptr, LBM_ENOMEM, "device allocation failed for a %d x %d x %d box", nx, ny, nz);
        release(h);
        return LBM_ENOMEM;
    }
    cudaError_t e = cudaMemsetAsync(h->ticket, 0, sizeof(unsigned) * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(unsigned) * 4, h->stream);
    if (e == cudaSuccess)
        e = lbm::launch_init(dim, prec, h->f[0], h->g[0], g, bc->T_init, bc->T_ref, bc->seed,
                             bc->perturb, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        fail(nullptr, LBM_ECUDA, "initialisation: %s", cudaGetErrorString(e));
        release(h);
        return LBM_ECUDA;
    }
    *out = h;
    return LBM_OK;
}

int lbm_destroy(lbm_handle h)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    release(h);
    return LBM_OK;
}

int lbm_set_stream(lbm_handle h, void* stream)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    h->stream = (cudaStream_t)stream;
    ++h->gen;
    return LBM_OK;
}

int lbm_set_omegas(lbm_handle h, const double* om_f, int n_f, const double* om_g, int n_g)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    if (om_f && n_f != h->qf) return fail(h, LBM_EINVAL, "expected %d flow rates, got %d", h->qf, n_f);
    if (om_g && n_g != h->qg) return fail(h, LBM_EINVAL, "expected %d energy rates, got %d", h->qg, n_g);
    for (int a = 0; om_f && a < n_f; ++a)
        if (!rate_ok(om_f[a])) return fail(h, LBM_EINVAL, "flow rate %d = %g outside (0, 2)", a, om_f[a]);
    for (int b = 0; om_g && b < n_g; ++b)
        if (!rate_ok(om_g[b])) return fail(h, LBM_EINVAL, "energy rate %d = %g outside (0, 2)", b, om_g[b]);
    for (int a = 0; om_f && a < n_f; ++a) h->hc.om_f[a] = om_f[a];
    for (int b = 0; om_g && b < n_g; ++b) h->hc.om_g[b] = om_g[b];
    ++h->gen;
    return LBM_OK;
}

int lbm_set_param(lbm_handle h, const char* key, double v)
{
    if (!h || !key) return fail(h, LBM_EINVAL, "handle or key is NULL");
    const std::string k(key);
    ++h->gen;
    if (k == "graph_steps") {
        const int v_i = (int)v;
        if (v != (double)v_i || v_i < 0 || v_i > 4096) return fail(h, LBM_EINVAL, "graph_steps must be an integer in [0, 4096]");
        h->graph_steps = v_i + (v_i & 1);
        return LBM_OK;
    }
    if (k == "block_x" || k == "block_y") {
        const int v_i = (int)v;
        if (v != (double)v_i || v_i < 1) return fail(h, LBM_EINVAL, "%s must be a positive integer", key);
        const int bx = k == "block_x" ? v_i : h->block_x, by = k == "block_y" ? v_i : h->block_y;
        if (bx != 0 && !(bx == 32 || bx == 64 || bx == 128 || bx == 256))
            return fail(h, LBM_EINVAL, "block_x must be 32, 64, 128 or 256");
        if (bx != 0 && by != 0 && bx * by > 256)
            return fail(h, LBM_EINVAL, "block_x * block_y must not exceed 256 threads");
        (k == "block_x" ? h->block_x : h->block_y) = v_i;
        if (h->block_x && !h->block_y) h->block_y = std::max(1, 256 / h->block_x);
        if (h->block_y && !h->block_x) h->block_x = 32;
        if (h->block_x * h->block_y > 256) h->block_y = 256 / h->block_x;
        if ((h->ny + h->block_y - 1) / h->block_y > 65535) {
            h->block_x = h->block_y = 0;
            return fail(h, LBM_EINVAL, "block_y too small for ny = %d", h->ny);
        }
        return LBM_OK;
    }
    if (k == "tma_rows") {
        const int v_i = (int)v;
        if (v != (double)v_i || !(v_i == 0 || v_i == 1 || v_i == 2 || v_i == 4))
            return fail(h, LBM_EINVAL, "tma_rows must be 0 (off), 1, 2 or 4");
        if (v_i == 0) {
            h->tma_rows = 0;
            return LBM_OK;
        }
        if (h->dim != 3 || h->prec == lbm::kF64)
            return fail(h, LBM_ENOTSUP, "the TMA-staged step covers the 3D FP32 and FP16S forms");
        const int eb = (int)lbm::storage_bytes(h->prec);
        for (int c = 0; c < 2; ++c) {
            std::string e;
            if (!lbm::make_tma_map(&h->tm[c].f, h->f[c], eb, h->nx, h->ny, h->nz, 27, v_i, &e) ||
                !lbm::make_tma_map(&h->tm[c].g, h->g[c], eb, h->nx, h->ny, h->nz, 15, v_i, &e))
                return fail(h, LBM_ENOTSUP, "%s", e.c_str());
            h->tm[c].ty = v_i;
        }
        h->tma_rows = v_i;
        return LBM_OK;
    }
    if (k == "index64") {
        if (!(v == 0.0 || v == 1.0)) return fail(h, LBM_EINVAL, "index64 must be 0 or 1");
        h->hc.index64 = (int)v;
        return LBM_OK;
    }
    if (k == "rows3d") {
        if (!(v == 0.0 || v == 1.0 || v == 2.0 || v == 4.0))
            return fail(h, LBM_EINVAL, "rows3d must be 0 (automatic), 1, 2 or 4");
        h->hc.rows3d = (int)v;
        return LBM_OK;
    }
    if (k == "adjoint_overlap") {
        if (!(v == 0.0 || v == 1.0)) return fail(h, LBM_EINVAL, "adjoint_overlap must be 0 or 1");
        h->adjoint_overlap = (int)v;
        return LBM_OK;
    }
    if (k == "adjoint_sync") {
        if (!(v == 0.0 || v == 1.0 || v == 2.0 || v == 3.0 || v == 4.0))
            return fail(h, LBM_EINVAL, "adjoint_sync must be 0 (64x2 blocks) or 1-4 (64x4, 128x2, 32x4, 64x2 with phase barriers)");
        h->hc.adj_sync = (int)v;
        return LBM_OK;
    }
    if (k == "fp16_stochastic") {
        if (!(v == 0.0 || v == 1.0)) return fail(h, LBM_EINVAL, "fp16_stochastic must be 0 or 1");
        h->hc.fp16_sr = (int)v;
        return LBM_OK;
    }
    if (k == "g_attractors") {
        if (!(v == 0.0 || v == 1.0)) return fail(h, LBM_EINVAL, "g_attractors must be 0 (option A) or 1 (option B)");
        h->hc.gopt = (int)v;
        return LBM_OK;
    }
    if (k == "adjoint_fp64") {
        if (!(v == 0.0 || v == 1.0)) return fail(h, LBM_EINVAL, "adjoint_fp64 must be 0 or 1");
        h->adjoint_arith = (int)v;
        return LBM_OK;
    }
    if (k == "adjoint_arith") {
        if (!(v == 0.0 || v == 1.0 || v == 2.0))
            return fail(h, LBM_EINVAL, "adjoint_arith must be 0 (FP32), 1 (FP64) or 2 (double-float)");
        h->adjoint_arith = (int)v;
        return LBM_OK;
    }
    if (k == "gbeta" || k == "T_ref") {
        if (!std::isfinite(v)) return fail(h, LBM_EINVAL, "%s must be finite", key);
        (k == "gbeta" ? h->hc.gbeta : h->hc.T_ref) = v;
        return LBM_OK;
    }
    if (!rate_ok(v)) return fail(h, LBM_EINVAL, "%s = %g outside (0, 2)", key, v);
    if (k == "omega_nu") {
        if (h->dim == 2) h->hc.om_f[4] = h->hc.om_f[5] = v;
        else h->hc.om_f[4] = h->hc.om_f[5] = h->hc.om_f[6] = h->hc.om_f[8] = h->hc.om_f[9] = v;
    } else if (k == "omega_alpha") {
        h->hc.om_g[1] = h->hc.om_g[2] = v;
        if (h->dim == 3) h->hc.om_g[3] = v;
    } else if (k == "omega_bulk") {
        h->hc.om_f[h->dim == 2 ? 3 : 7] = v;
    } else {
        return fail(h, LBM_EINVAL, "unknown parameter '%s'", key);
    }
    return LBM_OK;
}

int lbm_info(lbm_handle h, lbm_info_t* o)
{
    if (!h || !o) return fail(h, LBM_EINVAL, "handle or output is NULL");
    memset(o, 0, sizeof *o);
    o->lattice = h->lattice;
    o->precision = h->prec == lbm::kF64 ? LBM_FP64 : (h->prec == lbm::kF32 ? LBM_FP32 : LBM_FP16S);
    o->nx = h->nx;
    o->ny = h->ny;
    o->nz = h->nz;
    o->q_f = h->qf;
    o->q_g = h->qg;
    o->L = h->L;
    o->dT = h->dT;
    o->U = h->U;
    o->nu = h->nu;
    o->alpha = h->alpha;
    o->gbeta = h->hc.gbeta;
    o->T_ref = h->hc.T_ref;
    for (int a = 0; a < 27; ++a) o->om_f[a] = a < h->qf ? h->hc.om_f[a] : 0.0;
    for (int b = 0; b < 15; ++b) o->om_g[b] = b < h->qg ? h->hc.om_g[b] : 0.0;
    o->steps = h->steps;
    o->bytes_per_node_update = 2.0 * (h->qf + h->qg) * (double)lbm::storage_bytes(h->prec);
    o->state_bytes = kStateHeader + pop_bytes(h);
    const dim3 b = lbm::block_shape(h->nx, dim3(h->block_x, h->block_y, 1), h->dim);
    o->block_x = (int)b.x;
    o->block_y = (int)b.y;
    o->graph_steps = h->graph_steps;
    o->g_attractors = h->hc.gopt;
    o->fp16_stochastic = h->hc.fp16_sr;
    return LBM_OK;
}

// Capture graph_steps steps starting from buffer parity `par` into h->graph[par].
static int build_graph(lbm_s* h, int par)
{
    if (!h->capture_stream) LBM_CK(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    if (h->graph[par]) {
        LBM_CK(h, cudaGraphExecDestroy(h->graph[par]));
        h->graph[par] = nullptr;
    }
    cudaGraph_t g = nullptr;
    LBM_CK(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    int c = par;
    for (int t = 0; t < h->graph_steps && e == cudaSuccess; ++t) {
        e = lbm::launch_step(h->dim, h->prec, h->f[c], h->g[c], h->f[1 - c], h->g[1 - c], h->geo, h->hc,
                             h->status, dim3(h->block_x, h->block_y, 1), h->capture_stream,
                             h->tma_rows ? &h->tm[c] : nullptr);
        c = 1 - c;
    }
    const cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(h, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&h->graph[par], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
    h->graph_gen[par] = h->gen;
    return LBM_OK;
}

int lbm_step(lbm_handle h, long n)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    if (n < 0) return fail(h, LBM_EINVAL, "negative step count %ld", n);
    const lbm::NvtxRange range("lbm_step");
    // whole graphs of graph_steps steps, then single launches
    while (h->graph_steps > 0 && n >= h->graph_steps) {
        const int par = h->cur;
        if (!h->graph[par] || h->graph_gen[par] != h->gen) {
            const int rc = build_graph(h, par);
            if (rc) return rc;
        }
        LBM_CK(h, cudaGraphLaunch(h->graph[par], h->stream));
        h->steps += h->graph_steps;
        n -= h->graph_steps;
    }
    for (long t = 0; t < n; ++t) {
        const int c = h->cur;
        LBM_CK(h, lbm::launch_step(h->dim, h->prec, h->f[c], h->g[c], h->f[1 - c], h->g[1 - c],
                                   h->geo, h->hc, h->status, dim3(h->block_x, h->block_y, 1),
                                   h->stream, h->tma_rows ? &h->tm[c] : nullptr));
        h->cur = 1 - c;
        ++h->steps;
    }
    return LBM_OK;
}

int lbm_sync(lbm_handle h)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    unsigned st = 0;
    LBM_CK(h, cudaMemcpyAsync(&st, h->status, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    if (st) {
        LBM_CK(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
        if (st & 2u)
            return fail(h, LBM_ETIMEOUT, "a bounded wait of the TMA-staged step gave up by step %lld",
                        h->steps);
        return fail(h, LBM_EDIVERGED, "non-finite or non-positive density or temperature by step %lld",
                    h->steps);
    }
    return LBM_OK;
}

int lbm_fields(lbm_handle h, double* rho, double* ux, double* uy, double* uz, double* T,
               int device_ptrs)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    const size_t n = (size_t)h->geo.n;
    double* outs[5] = {rho, ux, uy, uz, T};
    if (device_ptrs) {   // the kernel writes the requested fields in place and skips the others
        LBM_CK(h, lbm::launch_fields(h->dim, h->prec, h->f[h->cur], h->g[h->cur], h->geo, h->hc, rho,
                                     ux, uy, uz, T, h->stream));
        return LBM_OK;
    }
    // host outputs: stage only the requested fields on the device
    int k_req = 0;
    for (int k = 0; k < 5; ++k) k_req += outs[k] != nullptr;
    if (k_req == 0) return LBM_OK;
    Tmp tmp(h, (size_t)k_req * n);
    if (!tmp.p) return fail(h, LBM_ENOMEM, "no device memory for the field staging buffer");
    double* dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int k = 0, m = 0; k < 5; ++k)
        if (outs[k]) dev[k] = tmp.p + (size_t)(m++) * n;
    LBM_CK(h, lbm::launch_fields(h->dim, h->prec, h->f[h->cur], h->g[h->cur], h->geo, h->hc, dev[0],
                                 dev[1], dev[2], dev[3], dev[4], h->stream));
    for (int k = 0; k < 5; ++k)
        if (outs[k])
            LBM_CK(h, cudaMemcpyAsync(outs[k], dev[k], n * sizeof(double), cudaMemcpyDeviceToHost,
                                      h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

static int nusselt_common(lbm_s* h, int face)
{
    if (face < 0 || face >= 2 * h->dim) return fail(h, LBM_EINVAL, "face %d is not a face of this box", face);
    if (h->geo.kind[face] != LBM_WALL_FIXED_T) return fail(h, LBM_EINVAL, "face %d is not a fixed-temperature wall", face);
    const int ext[3] = {h->nx, h->ny, h->nz};
    if (ext[face / 2] < 2) return fail(h, LBM_EINVAL, "fewer than two node layers normal to face %d", face);
    const double s = h->geo.T_wall[face] >= h->hc.T_ref ? 1.0 : -1.0;
    LBM_CK(h, lbm::launch_nusselt(h->dim, h->prec, h->f[h->cur], h->g[h->cur], h->geo, h->hc, face,
                                  -s * h->L / h->dT, h->nu_profile, h->nu_scratch, h->ticket,
                                  h->nu_result, h->stream));
    return LBM_OK;
}

int lbm_nusselt(lbm_handle h, int face, double* mean, double* nu_max, double* nu_min, int* j_max,
                int* j_min)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    int rc = nusselt_common(h, face);
    if (rc) return rc;
    double r[5];
    LBM_CK(h, cudaMemcpyAsync(r, h->nu_result, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    const long n = face_nodes(h, face);
    if (mean) *mean = r[0] / (double)n;
    if (nu_max) *nu_max = r[1];
    if (j_max) *j_max = (int)r[2];
    if (nu_min) *nu_min = r[3];
    if (j_min) *j_min = (int)r[4];
    return LBM_OK;
}

int lbm_nusselt_profile(lbm_handle h, int face, double* nu, long n, int device_ptrs)
{
    if (!h || !nu) return fail(h, LBM_EINVAL, "handle or output is NULL");
    int rc = nusselt_common(h, face);
    if (rc) return rc;
    if (n != face_nodes(h, face)) return fail(h, LBM_EINVAL, "face %d has %ld nodes, not %ld", face, face_nodes(h, face), n);
    LBM_CK(h, cudaMemcpyAsync(nu, h->nu_profile, n * sizeof(double),
                              device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_set_wall_profile(lbm_handle h, int face, const double* T_w, long n)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    if (face < 0 || face >= 2 * h->dim || h->geo.kind[face] != LBM_WALL_FIXED_T)
        return fail(h, LBM_EINVAL, "face %d is not a fixed-temperature wall", face);
    if (!T_w) {
        LBM_CK(h, cudaStreamSynchronize(h->stream));
        dev_free(h, h->profile[face]);
        h->profile[face] = nullptr;
        h->geo.profile[face] = nullptr;
        ++h->gen;
        return LBM_OK;
    }
    if (n != face_nodes(h, face)) return fail(h, LBM_EINVAL, "face %d has %ld nodes, not %ld", face, face_nodes(h, face), n);
    for (long k = 0; k < n; ++k)
        if (!std::isfinite(T_w[k])) return fail(h, LBM_EINVAL, "wall temperature %ld is not finite", k);
    if (!h->profile[face]) {
        h->profile[face] = (double*)dev_alloc(h, n * sizeof(double));
        if (!h->profile[face]) return fail(h, LBM_ENOMEM, "no device memory for the wall profile");
    }
    LBM_CK(h, cudaMemcpyAsync(h->profile[face], T_w, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    h->geo.profile[face] = h->profile[face];
    ++h->gen;
    return LBM_OK;
}

int lbm_adjoint_step(lbm_handle h, long n_steps, int objective_face, int design_face, double* J,
                     double* grad_Tw, long n)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    if (h->dim != 2) return fail(h, LBM_ENOTSUP, "the adjoint step is implemented for the D2Q9 pair");
    if (n_steps < 1) return fail(h, LBM_EINVAL, "n_steps must be at least 1");
    if (!J || !grad_Tw) return fail(h, LBM_EINVAL, "J or grad_Tw is NULL");
    for (int f : {objective_face, design_face})
        if (f < 0 || f >= 4 || h->geo.kind[f] != LBM_WALL_FIXED_T)
            return fail(h, LBM_EINVAL, "face %d is not a fixed-temperature wall of this box", f);
    if (objective_face == design_face) return fail(h, LBM_EINVAL, "objective and design face must differ");
    const int ext[2] = {h->nx, h->ny};
    if (ext[objective_face / 2] < 3) return fail(h, LBM_EINVAL, "fewer than three node layers normal to the objective face");
    if (n != face_nodes(h, design_face)) return fail(h, LBM_EINVAL, "design face %d has %ld nodes, not %ld", design_face, face_nodes(h, design_face), n);
    const lbm::NvtxRange range("lbm_adjoint_step");

    const size_t sb = lbm::storage_bytes(h->prec);
    const size_t fb = (size_t)h->qf * h->geo.n * sb, gb = (size_t)h->qg * h->geo.n * sb;
    const long K = (long)std::ceil(std::sqrt((double)n_steps));
    const long nck = (n_steps + K - 1) / K;
    // device memory: nck checkpoints, two sets of K segment states, two adjoint buffers, the
    // gradient.  Segment m's states are recomputed into one set while the adjoint steps of
    // segment m + 1 read the other (on a second stream, so the two overlap on the GPU).
    std::vector<void*> ckf(nck, nullptr), ckg(nck, nullptr);
    std::vector<void*> sgf_[2] = {std::vector<void*>(K, nullptr), std::vector<void*>(K, nullptr)};
    std::vector<void*> sgg_[2] = {std::vector<void*>(K, nullptr), std::vector<void*>(K, nullptr)};
    void* mu[2] = {nullptr, nullptr};
    double* grad = nullptr;
    const int arith = h->adjoint_arith;
    cudaGraphExec_t seg_exec[2] = {nullptr, nullptr};
    // the K adjoint steps of a full segment of set s starting on adjoint buffer a: adj_exec[s][a]
    cudaGraphExec_t adj_exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->stream);
        if (h->aux_stream) cudaStreamSynchronize(h->aux_stream);
        for (int s = 0; s < 2; ++s) {
            if (seg_exec[s]) cudaGraphExecDestroy(seg_exec[s]);
            for (int b = 0; b < 2; ++b)
                if (adj_exec[s][b]) cudaGraphExecDestroy(adj_exec[s][b]);
            if (ev_rec[s]) cudaEventDestroy(ev_rec[s]);
            if (ev_free[s]) cudaEventDestroy(ev_free[s]);
            for (auto p : sgf_[s]) dev_free(h, p);
            for (auto p : sgg_[s]) dev_free(h, p);
        }
        for (auto p : ckf) dev_free(h, p);
        for (auto p : ckg) dev_free(h, p);
        dev_free(h, mu[0]);
        dev_free(h, mu[1]);
        dev_free(h, grad);
    };
    bool ok = true;
    for (long m = 0; m < nck && ok; ++m) ok = (ckf[m] = dev_alloc(h, fb)) && (ckg[m] = dev_alloc(h, gb));
    // segment states 1 .. K-1, and state 0: the copy of a checkpoint that the recompute graph reads
    const bool seg_graph = K >= 3;
    // the second set only when another full segment precedes the last one
    const int nsets = seg_graph && nck >= 2 && h->adjoint_overlap ? 2 : 1;
    for (int s = 0; s < nsets; ++s)
        for (long r = seg_graph ? 0 : 1; r < K && ok; ++r)
            ok = (sgf_[s][r] = dev_alloc(h, fb)) && (sgg_[s][r] = dev_alloc(h, gb));
    const size_t mub = (size_t)(h->qf + h->qg) * h->geo.n * (arith == lbm::kAdjF32 ? sizeof(float) : 8);
    ok = ok && (mu[0] = dev_alloc(h, mub)) && (mu[1] = dev_alloc(h, mub)) &&
         (grad = (double*)dev_alloc(h, sizeof(double) * n));
    if (!ok) {
        cleanup();
        return fail(h, LBM_ENOMEM, "no device memory for %ld checkpoints of the adjoint", nck + K);
    }
#define ADJ_CK(expr)                                                                                \
    do {                                                                                            \
        cudaError_t e_ = (expr);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            cleanup();                                                                              \
            return fail(h, LBM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));                    \
        }                                                                                           \
    } while (0)
    const dim3 blk(h->block_x, h->block_y, 1);
    // forward pass with checkpoints s_0, s_K, s_2K, ...
    ADJ_CK(cudaMemcpyAsync(ckf[0], h->f[h->cur], fb, cudaMemcpyDeviceToDevice, h->stream));
    ADJ_CK(cudaMemcpyAsync(ckg[0], h->g[h->cur], gb, cudaMemcpyDeviceToDevice, h->stream));
    // (each segment through lbm_step, which replays its CUDA graphs)
    for (long m = 1; m <= nck; ++m) {
        const long len = std::min(m * K, n_steps) - (m - 1) * K;
        const int rc = lbm_step(h, len);
        if (rc) {
            cleanup();
            return rc;
        }
        if (m < nck) {
            ADJ_CK(cudaMemcpyAsync(ckf[m], h->f[h->cur], fb, cudaMemcpyDeviceToDevice, h->stream));
            ADJ_CK(cudaMemcpyAsync(ckg[m], h->g[h->cur], gb, cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    // objective at the final state
    const double sgn = h->geo.T_wall[objective_face] >= h->hc.T_ref ? 1.0 : -1.0;
    const double scale = -sgn * h->L / h->dT;
    ADJ_CK(lbm::launch_nusselt(h->dim, h->prec, h->f[h->cur], h->g[h->cur], h->geo, h->hc, objective_face,
                               scale, h->nu_profile, h->nu_scratch, h->ticket, h->nu_result, h->stream));
    double r[5];
    ADJ_CK(cudaMemcpyAsync(r, h->nu_result, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    // seed mu_{n+1} = dJ/dp_{n+1}
    int a = 0;
    ADJ_CK(cudaMemsetAsync(mu[a], 0, mub, h->stream));
    ADJ_CK(cudaMemsetAsync(grad, 0, sizeof(double) * n, h->stream));
    ADJ_CK(lbm::launch_adjoint_seed(h->geo, objective_face, scale, mu[a], arith, h->stream));
    // The K - 1 recompute steps of a full segment, state 0 -> 1 -> ... -> K - 1 of one set of
    // segment buffers, captured once per set as a CUDA graph; each full segment copies its
    // checkpoint into state 0 of its set and replays that set's graph.
    if (seg_graph) {
        if (!h->capture_stream) ADJ_CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
        for (int s = 0; s < nsets; ++s) {
            cudaGraph_t g = nullptr;
            ADJ_CK(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (long r2 = 1; r2 < K && e == cudaSuccess; ++r2)
                e = lbm::launch_step(h->dim, h->prec, sgf_[s][r2 - 1], sgg_[s][r2 - 1], sgf_[s][r2],
                                     sgg_[s][r2], h->geo, h->hc, h->status, blk, h->capture_stream);
            const cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &g);
            if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&seg_exec[s], g, 0);
            if (g) cudaGraphDestroy(g);
            ADJ_CK(e != cudaSuccess ? e : e2);
        }
    }
    if (nsets == 2) {
        if (!h->aux_stream) {
            // the lowest priority: the block scheduler prefers the adjoint steps' blocks
            int least = 0, greatest = 0;
            ADJ_CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
            ADJ_CK(cudaStreamCreateWithPriority(&h->aux_stream, cudaStreamNonBlocking, least));
        }
        for (int s = 0; s < 2; ++s) {
            ADJ_CK(cudaEventCreateWithFlags(&ev_rec[s], cudaEventDisableTiming));
            ADJ_CK(cudaEventCreateWithFlags(&ev_free[s], cudaEventDisableTiming));
        }
        // the aux stream starts after everything queued so far (checkpoints, seed)
        ADJ_CK(cudaEventRecord(ev_free[1], h->stream));
        ADJ_CK(cudaStreamWaitEvent(h->aux_stream, ev_free[1], 0));
    }
    // Recompute of full segment m into set s on stream st: its checkpoint into state 0, then the
    // set's graph.
    auto recompute_full = [&](long m, int s, cudaStream_t st) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(sgf_[s][0], ckf[m], fb, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sgg_[s][0], ckg[m], gb, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaGraphLaunch(seg_exec[s], st);
        return e;
    };
    // backward over the segments, last first; segment m uses set (nck - 1 - m) % 2
    for (long m = nck - 1; m >= 0; --m) {
        const int s = nsets == 2 ? (int)((nck - 1 - m) % 2) : 0;
        const long lo = m * K, hi = std::min((m + 1) * K, n_steps);
        std::vector<const void*> sf(hi - lo), sg(hi - lo);
        sf[0] = ckf[m];
        sg[0] = ckg[m];
        if (seg_graph && hi - lo == K) {
            if (m == nck - 1 || nsets == 1) ADJ_CK(recompute_full(m, s, h->stream));
            else ADJ_CK(cudaStreamWaitEvent(h->stream, ev_rec[s], 0));   // recomputed on the aux stream
            for (long r2 = 1; r2 < K; ++r2) {
                sf[r2] = sgf_[s][r2];
                sg[r2] = sgg_[s][r2];
            }
        } else {
            for (long r2 = 1; r2 < hi - lo; ++r2) {
                ADJ_CK(lbm::launch_step(h->dim, h->prec, sf[r2 - 1], sg[r2 - 1], sgf_[s][r2], sgg_[s][r2],
                                        h->geo, h->hc, h->status, blk, h->stream));
                sf[r2] = sgf_[s][r2];
                sg[r2] = sgg_[s][r2];
            }
        }
        // segment m - 1 (always full) into the other set, beside this segment's adjoint steps, once
        // the adjoint steps of segment m + 1, which read that set, are done
        if (nsets == 2 && m >= 1) {
            if (m + 1 <= nck - 1) ADJ_CK(cudaStreamWaitEvent(h->aux_stream, ev_free[1 - s], 0));
            ADJ_CK(recompute_full(m - 1, 1 - s, h->aux_stream));
            ADJ_CK(cudaEventRecord(ev_rec[1 - s], h->aux_stream));
        }
        if (seg_graph && hi - lo == K) {
            // a full segment: its K adjoint steps read state 0 of the set (the checkpoint's copy) and
            // states 1 .. K - 1, so they replay one graph per set and starting adjoint buffer,
            // captured on first use
            if (!adj_exec[s][a]) {
                cudaGraph_t g = nullptr;
                ADJ_CK(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = cudaSuccess;
                int b = a;
                for (long r2 = K - 1; r2 >= 0 && e == cudaSuccess; --r2) {
                    e = lbm::launch_adjoint_step_d2q9(h->prec, arith, sgf_[s][r2], sgg_[s][r2], mu[b],
                                                      mu[1 - b], h->geo, h->hc, design_face, grad,
                                                      h->capture_stream);
                    b = 1 - b;
                }
                const cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &g);
                if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&adj_exec[s][a], g, 0);
                if (g) cudaGraphDestroy(g);
                ADJ_CK(e != cudaSuccess ? e : e2);
            }
            ADJ_CK(cudaGraphLaunch(adj_exec[s][a], h->stream));
            if (K & 1) a = 1 - a;
        } else {
            for (long k = hi; k >= lo + 1; --k) {
                ADJ_CK(lbm::launch_adjoint_step_d2q9(h->prec, arith, sf[k - 1 - lo], sg[k - 1 - lo], mu[a],
                                                     mu[1 - a], h->geo, h->hc, design_face, grad,
                                                     h->stream));
                a = 1 - a;
            }
        }
        if (nsets == 2) ADJ_CK(cudaEventRecord(ev_free[s], h->stream));
    }
    ADJ_CK(cudaMemcpyAsync(grad_Tw, grad, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    ADJ_CK(cudaStreamSynchronize(h->stream));
#undef ADJ_CK
    *J = r[0] / (double)face_nodes(h, objective_face);
    cleanup();
    return LBM_OK;
}

int lbm_get_populations(lbm_handle h, double* f, double* g, int device_ptrs)
{
    if (!h || !f || !g) return fail(h, LBM_EINVAL, "handle or output is NULL");
    const size_t n = (size_t)h->geo.n;
    if (device_ptrs) {
        LBM_CK(h, lbm::launch_get_pops(h->dim, h->prec, h->f[h->cur], h->g[h->cur], h->geo, h->hc.T_ref,
                                       f, g, h->stream));
        return LBM_OK;
    }
    Tmp tmp(h, (h->qf + h->qg) * n);
    if (!tmp.p) return fail(h, LBM_ENOMEM, "no device memory for the staging buffer");
    LBM_CK(h, lbm::launch_get_pops(h->dim, h->prec, h->f[h->cur], h->g[h->cur], h->geo, h->hc.T_ref,
                                   tmp.p, tmp.p + h->qf * n, h->stream));
    LBM_CK(h, cudaMemcpyAsync(f, tmp.p, h->qf * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LBM_CK(h, cudaMemcpyAsync(g, tmp.p + h->qf * n, h->qg * n * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_set_populations(lbm_handle h, const double* f, const double* g, int device_ptrs)
{
    if (!h || !f || !g) return fail(h, LBM_EINVAL, "handle or input is NULL");
    const size_t n = (size_t)h->geo.n;
    if (device_ptrs) {
        LBM_CK(h, lbm::launch_set_pops(h->dim, h->prec, h->f[h->cur], h->g[h->cur], h->geo, h->hc.T_ref,
                                       f, g, h->stream));
        return LBM_OK;
    }
    Tmp tmp(h, (h->qf + h->qg) * n);
    if (!tmp.p) return fail(h, LBM_ENOMEM, "no device memory for the staging buffer");
    LBM_CK(h, cudaMemcpyAsync(tmp.p, f, h->qf * n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    LBM_CK(h, cudaMemcpyAsync(tmp.p + h->qf * n, g, h->qg * n * sizeof(double), cudaMemcpyHostToDevice,
                              h->stream));
    LBM_CK(h, lbm::launch_set_pops(h->dim, h->prec, h->f[h->cur], h->g[h->cur], h->geo, h->hc.T_ref,
                                   tmp.p, tmp.p + h->qf * n, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_get_state(lbm_handle h, void* buf, size_t bytes)
{
    if (!h || !buf) return fail(h, LBM_EINVAL, "handle or buffer is NULL");
    if (bytes != kStateHeader + pop_bytes(h)) return fail(h, LBM_EINVAL, "state needs %zu bytes, got %zu", kStateHeader + pop_bytes(h), bytes);
    unsigned long long hdr[8] = {kStateMagic, (unsigned long long)h->lattice, (unsigned long long)h->prec,
                                 (unsigned long long)h->nx, (unsigned long long)h->ny,
                                 (unsigned long long)h->nz, (unsigned long long)h->steps, 0ULL};
    memcpy(buf, hdr, sizeof hdr);
    char* p = (char*)buf + kStateHeader;
    const size_t fb = (size_t)h->qf * h->geo.n * lbm::storage_bytes(h->prec);
    const size_t gb = (size_t)h->qg * h->geo.n * lbm::storage_bytes(h->prec);
    LBM_CK(h, cudaMemcpyAsync(p, h->f[h->cur], fb, cudaMemcpyDeviceToHost, h->stream));
    LBM_CK(h, cudaMemcpyAsync(p + fb, h->g[h->cur], gb, cudaMemcpyDeviceToHost, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_set_state(lbm_handle h, const void* buf, size_t bytes)
{
    if (!h || !buf) return fail(h, LBM_EINVAL, "handle or buffer is NULL");
    if (bytes != kStateHeader + pop_bytes(h)) return fail(h, LBM_EINVAL, "state needs %zu bytes, got %zu", kStateHeader + pop_bytes(h), bytes);
    unsigned long long hdr[8];
    memcpy(hdr, buf, sizeof hdr);
    if (hdr[0] != kStateMagic || hdr[1] != (unsigned long long)h->lattice ||
        hdr[2] != (unsigned long long)h->prec || hdr[3] != (unsigned long long)h->nx ||
        hdr[4] != (unsigned long long)h->ny || hdr[5] != (unsigned long long)h->nz)
        return fail(h, LBM_EINVAL, "checkpoint does not match this box (lattice, precision or shape)");
    const char* p = (const char*)buf + kStateHeader;
    const size_t fb = (size_t)h->qf * h->geo.n * lbm::storage_bytes(h->prec);
    const size_t gb = (size_t)h->qg * h->geo.n * lbm::storage_bytes(h->prec);
    LBM_CK(h, cudaMemcpyAsync(h->f[h->cur], p, fb, cudaMemcpyHostToDevice, h->stream));
    LBM_CK(h, cudaMemcpyAsync(h->g[h->cur], p + fb, gb, cudaMemcpyHostToDevice, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    h->steps = (long long)hdr[6];
    return LBM_OK;
}

}  // extern "C"
