// kernels.h -- host-side launchers of the CUDA kernels (internal to liblbm.so).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#include <nvtx3/nvToolsExt.h>

#include "lbm_common.cuh"
#include "../../include/lbm.h"
#include <string>

namespace lbm {

// A named NVTX range on the calling thread's timeline for the duration of a library call
// (lbm_step, lbm_batch_step, lbm_adjoint_step): profilers that record NVTX show it above the
// kernels the call queued; without such a tool attached it costs two calls into a stub.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

enum Prec { kF64 = 0, kF32 = 1, kF16S = 2 };

// Relaxation rates and coupling in double precision; converted to the kernel's register type.
struct HostCoeffs {
    double om_f[27];
    double om_g[15];
    double gbeta, T_ref;
    int gaxis;
    int gopt;   // energy attractors of orders 3-4: 0 = option A, 1 = option B
    int fp16_sr;   // F16S storage: stochastic (1) or nearest (0) rounding of stored deviations
    int index64;   // 1: the step uses 64-bit element offsets even where 32-bit ones suffice
    int rows3d;    // 3D FP32 / FP16S step: rows of its column each thread updates (1, 2 or 4; 0 automatic)
    int adj_sync;  // adjoint step blocks: 0 = 64x2; with phase barriers 1 = 64x4, 2 = 128x2 (default),
                   // 3 = 32x4, 4 = 64x2
};

size_t storage_bytes(int prec);

// A validated box and its derived parameters (plan_box in api.cu).
struct BoxPlan {
    int lattice, prec, dim, nx, ny, nz, qf, qg;
    Geometry geo;
    HostCoeffs hc;
    double L, dT, U, nu, alpha;
};
int plan_box(int lattice, int nx, int ny, int nz, double Ra, double Pr, double Ma, const lbm_bc* bc,
             BoxPlan* P, std::string* err);
// Records the message of a failed call that has no handle (lbm_create, lbm_nusselt_static); lbm_last_error(NULL)
// returns it on the calling thread.  Returns code.
int fail_no_handle(int code, const char* fmt, ...);
// The process-wide device allocator hooks of lbm_set_allocator.
void current_allocator(lbm_alloc_fn* a, lbm_free_fn* f, void** ctx);

// Tensor maps of the input buffers of a TMA-staged 3D step (step_d3q27_tma.cuh) and its tile
// height (1, 2 or 4 rows of 64 nodes).
struct TmaMaps {
    CUtensorMap f, g;
    int ty;
};
// Encode the 4D map (x, y, z, plane) of one population buffer with boxes of (64 + 32 / elem_bytes)
// x ty x 1 x 1 elements.
// Fails (returns false, with a message) when the x stride is not a multiple of 16 bytes.
bool make_tma_map(CUtensorMap* out, void* base, int elem_bytes, int nx, int ny, int nz, int planes,
                  int ty, std::string* err);

// block: thread-block shape of the step launch (x-major); block.x == 0 selects the default.
// tma: tensor maps of fin / gin for the TMA-staged 3D step (FP32 and FP16S), or nullptr.
cudaError_t launch_step(int dim, int prec, const void* fin, const void* gin, void* fout, void* gout,
                        const Geometry& geo, const HostCoeffs& hc, unsigned* status, dim3 block,
                        cudaStream_t st, const TmaMaps* tma = nullptr);
cudaError_t launch_step_d3q27_tma_f32(const TmaMaps& tm, const void* fin, const void* gin, void* fout,
                                      void* gout, const Geometry& geo, const HostCoeffs& hc,
                                      unsigned* status, cudaStream_t st);
cudaError_t launch_step_d3q27_tma_f16s(const TmaMaps& tm, const void* fin, const void* gin, void* fout,
                                       void* gout, const Geometry& geo, const HostCoeffs& hc,
                                       unsigned* status, cudaStream_t st);
cudaError_t launch_step_d2q9(int prec, const void* fin, const void* gin, void* fout, void* gout,
                             const Geometry& geo, const HostCoeffs& hc, unsigned* status,
                             dim3 block, cudaStream_t st);
cudaError_t launch_step_d3q27_f64(const void* fin, const void* gin, void* fout, void* gout,
                                  const Geometry& geo, const HostCoeffs& hc, unsigned* status,
                                  dim3 block, cudaStream_t st);
cudaError_t launch_step_d3q27_f32(const void* fin, const void* gin, void* fout, void* gout,
                                  const Geometry& geo, const HostCoeffs& hc, unsigned* status,
                                  dim3 block, cudaStream_t st);
cudaError_t launch_step_d3q27_f16s(const void* fin, const void* gin, void* fout, void* gout,
                                   const Geometry& geo, const HostCoeffs& hc, unsigned* status,
                                   dim3 block, cudaStream_t st);

cudaError_t launch_init(int dim, int prec, void* f, void* g, const Geometry& geo, double T_init,
                        double T_ref, uint64_t seed, double perturb, cudaStream_t st);
cudaError_t launch_fields(int dim, int prec, const void* f, const void* g, const Geometry& geo,
                          const HostCoeffs& hc, double* rho, double* ux, double* uy, double* uz,
                          double* T, cudaStream_t st);
cudaError_t launch_get_pops(int dim, int prec, const void* f, const void* g, const Geometry& geo,
                            double T_ref, double* fo, double* go, cudaStream_t st);
cudaError_t launch_set_pops(int dim, int prec, void* f, void* g, const Geometry& geo, double T_ref,
                            const double* fi, const double* gi, cudaStream_t st);

// Local wall Nusselt numbers of a fixed-T face and their mean / max / min.
// scratch must hold nusselt_scratch_doubles(n_face) doubles plus one unsigned ticket (ticket
// must be zero on entry and is left zero on exit).  result receives
// {sum, max, argmax, min, argmin} as doubles.
size_t nusselt_scratch_doubles(long n_face);
cudaError_t launch_nusselt(int dim, int prec, const void* f, const void* g, const Geometry& geo,
                           const HostCoeffs& hc, int face, double scale, double* profile,
                           double* scratch, unsigned* ticket, double* result, cudaStream_t st);

// Adjoint of the D2Q9 step (adjoint_d2q9.cuh): seed mu_{n+1} = dJ/dp for J = mean Nu on `face`
// (mu must be zeroed first), and one fused adjoint step mu_{k+1} -> mu_k from the state s_{k-1},
// adding the design-face wall-temperature gradient (FP64) to grad.  `arith` is the arithmetic of
// the vector-Jacobian products and of mu: FP32 (4-byte mu), FP64 or double-float (8-byte mu).
enum AdjointArith { kAdjF32 = 0, kAdjF64 = 1, kAdjDF = 2 };
cudaError_t launch_adjoint_seed(const Geometry& geo, int face, double scale, void* mu, int arith,
                                cudaStream_t st);
cudaError_t launch_adjoint_step_d2q9(int prec, int arith, const void* f_prev, const void* g_prev,
                                     const void* mu_in, void* mu_out, const Geometry& geo,
                                     const HostCoeffs& hc, int design_face, double* grad,
                                     cudaStream_t st);

}  // namespace lbm

namespace lbm {

template <class R, int QF, int QG>
inline Coeffs<R, QF, QG> make_coeffs(const HostCoeffs& h)
{
    Coeffs<R, QF, QG> c{};
    for (int a = 0; a < QF; ++a) {
        c.om_f[a] = R(h.om_f[a]);
        c.hf[a] = R(1.0 - 0.5 * h.om_f[a]);
    }
    for (int b = 0; b < QG; ++b) c.om_g[b] = R(h.om_g[b]);
    c.gbeta = R(h.gbeta);
    c.T_ref = R(h.T_ref);
    c.gaxis = h.gaxis;
    c.gopt = h.gopt;
    c.fp16_sr = h.fp16_sr;
    return c;
}

// Default thread blocks, x-major so that a warp reads and writes 32 consecutive nodes; a
// caller-chosen shape (block.x > 0) replaces it.  2D: 256 threads.  3D: 64 x 1, which at 96
// registers per thread lets 10 blocks (20 warps) share an SM against 16 warps for 256-thread
// blocks (measured on the 256^3 cavity: 16.4 vs 15.8 GLUPS).
inline dim3 block_shape(int nx, dim3 chosen = dim3(0, 0, 0), int dim = 2)
{
    if (chosen.x > 0) return dim3(chosen.x, chosen.y, 1);
    if (dim == 3) return dim3(nx > 32 ? 64 : 32, 1, 1);
    const int bx = nx >= 128 ? 128 : ((nx + 31) / 32) * 32;
    return dim3(bx, 256 / bx, 1);
}

// 32-bit element offsets suffice when every population plane index q * n fits in 32 bits.
inline bool index32(const Geometry& g, int q)
{
    return (unsigned long long)q * (unsigned long long)g.n <= 0xffffffffULL;
}

// The step's offset width: 32-bit where q n < 2^32, unless the handle forces the 64-bit
// instantiation (which boxes above that size run; forcing it lets small boxes test it).
inline bool step_index32(const Geometry& g, int q, const HostCoeffs& hc)
{
    return index32(g, q) && !hc.index64;
}

// The energy rates are those lbm_create sets (option A; every rate 1 except the first-order ones,
// which carry alpha), so the 3D step may take the unit-rate energy collision.
inline bool unit_energy_rates(const HostCoeffs& h)
{
    if (h.gopt != 0) return false;
    for (int b = 4; b < 15; ++b)
        if (h.om_g[b] != 1.0) return false;
    return true;
}

// The 3D flow rates are those lbm_create sets: every rate 1 except the shear rates (slots 4-6,
// 8, 9), the bulk rate (slot 7) included.
inline bool unit_flow_rates(const HostCoeffs& h)
{
    for (int a = 0; a < 27; ++a)
        if (!(a >= 4 && a <= 6) && a != 8 && a != 9 && h.om_f[a] != 1.0) return false;
    return true;
}

// Which collision instance the 3D step takes: 0 general, 1 unit-rate energy collision, 2 that and
// the unit-rate flow relaxation.
inline int rate_class(const HostCoeffs& h)
{
    if (!unit_energy_rates(h)) return 0;
    return unit_flow_rates(h) ? 2 : 1;
}

// Rows per thread of the 3D FP32 / FP16S step: the handle's setting, or when that is 0 the faster
// one measured on the 256^3 cavity: one for FP16S storage with the reduced collisions of the
// default rates (+0.8 % against two), two otherwise (FP32 +1.2 % at its 72 registers; FP16S with
// the general collision +0.5-0.9 %).
inline int rows3d_for(const HostCoeffs& h, bool f16s)
{
    if (h.rows3d > 0) return h.rows3d;
    return f16s && rate_class(h) == 2 ? 1 : 2;
}

inline dim3 grid_shape(const Geometry& g, dim3 b)
{
    return dim3((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y, g.nz);
}

}  // namespace lbm
