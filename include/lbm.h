/*
 * lbm.h -- C ABI of liblbm.so: the GB300 (sm_103a) hot path of the Fokker-Planck central-moment
 * lattice Boltzmann method for thermal convection (Schupbach & Premnath, arXiv 2504.09041).
 *
 * One time step advances two coupled lattices at every node: the flow populations f (D2Q9,
 * App. A; or D3Q27, Sec. 5.1-5.2) relaxed toward the FP central-moment attractors with the
 * renormalized diffusion tensor and the Boussinesq source, and the energy populations g (D2Q9,
 * App. B; or D3Q15, App. C) relaxed toward their own (option-A) attractors.  The step is one fused
 * pull-stream + collide kernel launch (Eqs. LBMsteps-collide / LBMsteps-stream).
 *
 * Conventions used by every entry point:
 *  - Return value: LBM_OK (0) or one of the lbm_status codes; nothing traps, no exception crosses
 *    the ABI.  lbm_last_error(h) describes the most recent failure on h (or, when h is NULL,
 *    of a call without a handle on the calling thread).
 *  - Node index i = x + nx * (y + ny * z), x fastest.  Population arrays are [q][nz][ny][nx] in
 *    the paper's link order (D2Q9 Eqs. ex, ey; D3Q27 Sec. 5.2; D3Q15 Sec. 5.4).
 *  - Faces are numbered 0..5 = -x, +x, -y, +y, -z, +z.  2D boxes have nz = 1 and ignore the z faces.
 *  - The library owns its device buffers (allocated through lbm_set_allocator's hook, cudaMalloc by
 *    default).  Caller buffers are only read or written during the call that receives them.
 *  - Work is queued on the handle's stream (lbm_set_stream; the legacy default stream otherwise).
 *    Calls that return data to the host synchronize that stream.
 *  - Handles are not thread-safe; use one handle per thread or serialize calls.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_s* lbm_handle;

enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = 1,     /* invalid argument (bad size, face, key, rate outside (0, 2), ...) */
    LBM_ENOMEM = 2,     /* the device allocator returned NULL */
    LBM_ECUDA = 3,      /* a CUDA call failed; lbm_last_error has the CUDA message */
    LBM_EDIVERGED = 4,  /* a node saw a non-finite or non-positive density or a non-finite T */
    LBM_ETIMEOUT = 5,   /* a bounded device-side wait gave up (the kernel returned, no hang) */
    LBM_ENOTSUP = 6     /* valid request that this library does not support */
};

/* Lattice pair, OR-ed with one storage precision. */
enum lbm_lattice { LBM_D2Q9_D2Q9 = 1, LBM_D3Q27_D3Q15 = 2 };
enum lbm_prec {
    LBM_FP64 = 0x000,   /* populations stored and relaxed in FP64 */
    LBM_FP32 = 0x100,   /* populations stored and relaxed in FP32 */
    LBM_FP16S = 0x200   /* FP16 storage of f_a - w_a and g_a - w_a T_o, FP32 moment algebra */
};
enum lbm_face_bc {
    LBM_PERIODIC = 0,        /* both faces of an axis must be periodic, or neither */
    LBM_WALL_ADIABATIC = 1,  /* half-way bounce-back of f (no slip) and of g (zero heat flux) */
    LBM_WALL_FIXED_T = 2     /* bounce-back of f, anti-bounce-back of g at T_wall (Sec. 6.1) */
};

typedef struct {
    int face[6];                /* lbm_face_bc of -x, +x, -y, +y, -z, +z */
    double T_wall[6];           /* wall temperature of LBM_WALL_FIXED_T faces */
    double T_init;              /* initial uniform temperature */
    double T_ref;               /* T_o of the Boussinesq force F = g beta (T - T_o) (Sec. 6.1) */
    int gravity_axis;           /* axis of the buoyancy force: 1 (y) in 2D, 2 (z) in 3D */
    unsigned long long seed;    /* splitmix64 seed of the initial temperature perturbation */
    double perturb;             /* T_init += perturb * (2 U_i - 1), U_i uniform in [0, 1) */
} lbm_bc;

typedef struct {
    int lattice, precision;     /* lbm_lattice and lbm_prec values */
    int nx, ny, nz, q_f, q_g;
    double L;                   /* characteristic length: nodes across the fixed-T faces' axis */
    double dT;                  /* T_H - T_C over the fixed-T faces (1 if fewer than two differ) */
    double U, nu, alpha, gbeta; /* U_o = Ma/sqrt(3); nu = U L sqrt(Pr/Ra); alpha = nu/Pr;
                                   g beta = U^2/(L dT)   (Sec. 6.1, Sec. 7) */
    double T_ref;
    double om_f[27], om_g[15];  /* relaxation rates in use (see lbm_set_omegas) */
    long long steps;            /* time steps taken since creation */
    double bytes_per_node_update; /* algorithmic HBM bytes per node and step: 2 (q_f + q_g) size */
    size_t state_bytes;         /* size of an lbm_get_state checkpoint */
    int block_x, block_y;       /* thread-block shape of the step launch */
    int graph_steps;            /* steps per CUDA graph replayed by lbm_step (0: plain launches) */
    int g_attractors;           /* energy attractors of orders 3-4: 0 = option A, 1 = option B */
    int fp16_stochastic;        /* LBM_FP16S: 1 = stochastic rounding of the stored deviations */
} lbm_info_t;

/*
 * Device allocator hook (process-wide).  alloc(bytes, ctx) returns device memory or NULL;
 * free(ptr, ctx) releases it.  NULL functions restore cudaMalloc / cudaFree.  A handle keeps the
 * hook it was created with.  Returns LBM_OK.
 */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* ctx);
typedef void (*lbm_free_fn)(void* ptr, void* ctx);
LBM_API int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void* ctx);

/*
 * Create a box of nx * ny * nz nodes (nz = 1 for LBM_D2Q9_D2Q9) for the cavity problems of
 * Sec. 6.1 / 6.2: Rayleigh number Ra, Prandtl number Pr and Mach number Ma = sqrt(3) U_o
 * (Sec. 7) fix nu, alpha and g beta (see lbm_info_t) and the rates
 *   nu = c_s^2 (1/omega - 1/2)        on the shear moments of f (App. A: omega_4, omega_5),
 *   alpha = c_s^2 (1/omega - 1/2)     on the first-order moments of g (App. B, App. C),
 * every other rate 1.0 (App. A, B, C).  The populations start at the rest attractors at density 1
 * and temperature T_init (+ the seeded perturbation).
 * Errors: LBM_EINVAL (sizes < 1, nz != 1 in 2D, more than 2^31 - 1 nodes, Ra/Pr/Ma not positive
 * and finite, bad face kinds, one-sided periodic axis, bad gravity axis), LBM_ENOMEM, LBM_ECUDA.
 * On success *out owns the handle; release it with lbm_destroy.
 */
LBM_API int lbm_create(int lattice, int nx, int ny, int nz, double Ra, double Pr, double Ma,
               const lbm_bc* bc, lbm_handle* out);
LBM_API int lbm_destroy(lbm_handle h);

/* Queue all further work of h on the CUDA stream `stream` (a cudaStream_t; NULL = legacy). */
LBM_API int lbm_set_stream(lbm_handle h, void* stream);

/*
 * Replace the relaxation rates.  om_f: n_f = q_f rates of the flow collision; om_g: n_g = q_g
 * rates of the energy collision (either pointer may be NULL to keep the current rates).
 *  - D2Q9 f: omega_0..omega_8 of App. A Step 3 (omega_3 on kappa_2s, omega_4 on kappa_2d).
 *  - D2Q9 g: omega_0..omega_8 of App. B Step 3 (omega_3, omega_4 on the eta_2s, eta_2d pair).
 *  - D3Q15 g: omega_0..omega_14 of App. C Step 3.
 *  - D3Q27 f: one rate per entry of the central-moment vector of Sec. 5.2, except slot 7 which
 *    relaxes the trace kappa_200 + kappa_020 + kappa_002 and slots 8, 9 which relax the deviators
 *    kappa_200 - kappa_020 and kappa_200 - kappa_002.
 * Every rate must lie in (0, 2) (App. A).  Errors: LBM_EINVAL.
 */
LBM_API int lbm_set_omegas(lbm_handle h, const double* om_f, int n_f, const double* om_g, int n_g);

/* Set a scalar parameter: "gbeta", "T_ref", "omega_nu", "omega_alpha", "omega_bulk",
 * "g_attractors" (0: option A, Eqs. MvT2D / g-attractorsD3Q15optionA, the default and the paper's
 * choice; 1: option B, the renormalized energy attractors of orders 3-4 of Eq. MvT2DoptionB and
 * its D3Q15 counterpart in Sec. 5.3, with D-hat' = eta~ / T from the post-collision second
 * moments), "fp16_stochastic" (LBM_FP16S storage: 1, the default, rounds each stored deviation
 * stochastically, up or down with probabilities that make the rounding unbiased, so that updates
 * smaller than half an FP16 step accumulate in expectation; 0 rounds to nearest), "adjoint_arith" (arithmetic of lbm_adjoint_step's vector-Jacobian products and adjoint state: 2, the default, double-float, i.e. pairs of FP32
 * numbers with a 48-bit significand evaluated on the FP32 pipes; 1 FP64; 0 FP32), "adjoint_fp64" (0 or 1: the same as "adjoint_arith" 0 or 1),
 * "adjoint_sync" (thread blocks of the adjoint kernel: 0 = 64 x 2; 1-4 = 64 x 4, 128 x 2 (the
 * default), 32 x 4, 64 x 2 whose warps pass a barrier between the phases of the node's work so
 * that they share the instruction fetches of the long unrolled product; results agree to
 * rounding), "adjoint_overlap" (1, the default: lbm_adjoint_step recomputes the next segment's
 * states on a second, low-priority stream while the adjoint steps of the current one run, with
 * a second set of segment buffers; 0: one stream, one set),
 * "graph_steps" (even count of steps that lbm_step replays as one CUDA graph; 0 disables),
 * "rows3d" (1, 2 or 4: rows of its column that each thread of the 3D FP32 / FP16S step updates
 * in turn; 0, the default: the faster count measured for the storage and rates, one for FP16S
 * with the default rates and two otherwise; results are bitwise the same),
 * "index64" (1: the step kernels use 64-bit element offsets, the instantiation that boxes with
 * q n >= 2^32 run, on any box; results are bitwise those of the 32-bit form; for testing that path), or the
 * thread-block shape of the step launch, "block_x" (32, 64, 128 or 256) and "block_y"
 * (block_x * block_y <= 256), or "tma_rows" (0 = off; 1, 2 or 4: the 3D FP32 / FP16S step stages
 * its pull through shared memory with tensor copies in tiles of 64 x tma_rows nodes; results are
 * bitwise those of the plain step; needs nx times the element size to be a multiple of 16 bytes,
 * else LBM_ENOTSUP).  Errors: LBM_EINVAL for an unknown key, a rate outside (0, 2) or a
 * bad block shape. */
LBM_API int lbm_set_param(lbm_handle h, const char* key, double value);
LBM_API int lbm_info(lbm_handle h, lbm_info_t* out);

/*
 * Advance n >= 0 time steps (asynchronous on the handle's stream).  Runs of graph_steps steps (32 by
 * default) are replayed from a CUDA graph captured once per buffer parity and launch settings;
 * the rest are plain launches.  Per step one fused launch that
 * pulls the post-collision populations along every link with the wall rules of Sec. 6.1, forms
 * T = sum g, F = g beta (T - T_o) along gravity, rho = sum f, rho u = sum f e + F/2 (App. A Step 7),
 * and relaxes f and g in central-moment space (App. A/B/C Steps 1-5).
 * Errors: LBM_EINVAL (n < 0), LBM_ECUDA (launch failure).  Divergence is reported by lbm_sync.
 */
LBM_API int lbm_step(lbm_handle h, long n);

/* Wait for the handle's queued work and report divergence: LBM_EDIVERGED if any node of any step
 * since the last lbm_sync saw a non-finite or non-positive density or a non-finite temperature. */
LBM_API int lbm_sync(lbm_handle h);

/*
 * Macroscopic fields of the streamed populations at the current time (App. A Step 7 and App. B/C
 * Step 7): rho, u (with the half-force term) and T, FP64, n = nx*ny*nz values each.  The sums over
 * the links run in the register type of the storage (FP32 for FP32 and FP16 storage) and are
 * promoted to FP64.  Pointers are device pointers when device_ptrs != 0, else host pointers; any
 * pointer may be NULL, and only the requested fields are computed and copied.
 */
LBM_API int lbm_fields(lbm_handle h, double* rho, double* ux, double* uy, double* uz, double* T,
               int device_ptrs);

/*
 * Wall Nusselt number on a fixed-temperature face (Sec. 6.1): at every wall node,
 *   dT/dn = -8/3 T_w + 3 T_1 - 1/3 T_2   (wall at 0, node layers at 1/2 and 3/2, n into the fluid)
 *   Nu = -s (L / dT) dT/dn,  s = +1 if the face's T_wall >= T_ref, else -1,
 * reduced in FP64 to the mean over the face nodes and the max / min with their tangential node
 * index j (x faces: j = y + ny z; y faces: j = x + nx z; z faces: j = x + nx y; its location is
 * (j + 1/2) / N along that axis).  Any output pointer may be NULL.
 * Errors: LBM_EINVAL (face not a fixed-T wall of this box, or fewer than 2 node layers).
 */
LBM_API int lbm_nusselt(lbm_handle h, int face, double* mean, double* nu_max, double* nu_min, int* j_max,
                int* j_min);
/* The local Nu of every node of that face (n = number of face nodes), host or device pointer. */
LBM_API int lbm_nusselt_profile(lbm_handle h, int face, double* nu, long n, int device_ptrs);

/* Per-node wall temperature of a fixed-T face (n = face nodes, tangential order as above, host
 * pointer); T_w = NULL returns the face to its uniform T_wall.  The profile enters the
 * half-way anti-bounce-back of Sec. 6.1, g_abar = -g~_a + 2 w_a T_w(j), on every link that crosses
 * the face at node j, and the wall value of the Nusselt derivative there.  Errors: LBM_EINVAL. */
LBM_API int lbm_set_wall_profile(lbm_handle h, int face, const double* T_w, long n);

/*
 * Reverse-mode gradient of a wall Nusselt objective with respect to a wall-temperature profile.
 * J = the mean Nu on objective_face (as lbm_nusselt) after n_steps >= 1 steps from the current
 * state; grad_Tw[j] = dJ/dT_w(j) for every node j of design_face (a fixed-T face other than
 * objective_face; tangential order as in lbm_set_wall_profile).  The call runs the n_steps forward
 * (the handle ends at that state, as after lbm_step), keeping a checkpoint every
 * K = ceil(sqrt(n_steps)) steps, then n_steps fused adjoint steps backward, recomputing each
 * segment of K states once from its checkpoint: about 2 sqrt(n_steps) states of device memory and
 * one extra forward pass.  The vector-Jacobian products of the collision are evaluated at the
 * recomputed forward intermediates of each node (in the forward step's own register type, FP32
 * for FP32 / FP16 states), with the adjoint carried in double-float arithmetic by default: the
 * gradient equals the FP64 adjoint's to about 1e-11 relative, at a third of its cost on GPUs whose
 * FP64 rate is a small fraction of their FP32 rate.  lbm_set_param "adjoint_arith" = 1 selects FP64, 0 FP32 (about twice as fast
 * again, gradients to about 1e-4 relative after 2000 steps).  The design gradient is always
 * accumulated in FP64.  2D (D2Q9 pair) only.
 * J and grad_Tw are host pointers; n must equal the number of design-face nodes.
 * Errors: LBM_EINVAL (bad faces, n, n_steps), LBM_ENOTSUP (3D), LBM_ENOMEM, LBM_ECUDA.
 */
LBM_API int lbm_adjoint_step(lbm_handle h, long n_steps, int objective_face, int design_face,
                             double* J, double* grad_Tw, long n);

/*
 * The stored state is the post-collision populations of the last step (before streaming).
 * lbm_get_populations / lbm_set_populations convert it from / to FP64 arrays f[q_f][n],
 * g[q_g][n] (device pointers when device_ptrs != 0).  With FP16S storage the values are
 * shift + deviation, formed in FP64.
 */
LBM_API int lbm_get_populations(lbm_handle h, double* f, double* g, int device_ptrs);
LBM_API int lbm_set_populations(lbm_handle h, const double* f, const double* g, int device_ptrs);

/* Checkpoint / restart in the storage format: bytes must equal lbm_info's state_bytes; buf is a
 * host buffer.  lbm_set_state also restores the step counter.  Errors: LBM_EINVAL on a size,
 * lattice, precision or shape mismatch. */
LBM_API int lbm_get_state(lbm_handle h, void* buf, size_t bytes);
LBM_API int lbm_set_state(lbm_handle h, const void* buf, size_t bytes);

/* The message of the most recent failure on h; with h = NULL, that of the most recent failed
 * call without a handle (lbm_create, lbm_nusselt_static) on the calling thread. */
LBM_API const char* lbm_last_error(lbm_handle h);
LBM_API const char* lbm_status_string(int status);

/*
 * Self-test of the bounded device waits (the TMA-staged step's mbarrier waits use the same code).
 * One thread waits on a shared-memory mbarrier that nothing arrives on, for at most `seconds`
 * (0 < seconds <= 10, converted with the device's clock rate), then records the timeout and
 * returns.  The paper has no counterpart: it lets the failure path of a device wait be tested
 * without hanging a GPU.  *timed_out receives 1 when the wait gave up (the expected outcome).
 * Returns LBM_ETIMEOUT in that case, LBM_OK if the wait completed, LBM_EINVAL for a bad argument,
 * LBM_ENOMEM or LBM_ECUDA on errors.  Runs on, and synchronizes, the legacy default stream.
 */
LBM_API int lbm_probe_bounded_wait(double seconds, int* timed_out);

/*
 * Wall Nusselt reduction that allocates nothing.  The paper has no counterpart: this is the
 * lbm_nusselt computation offered to callers that may not allocate device memory.  Such callers
 * own all of their device memory through another allocator (a framework's caching pool, or a
 * fixed budget reserved at start-up); a cudaMalloc issued behind their back by a library would
 * fail or break their accounting.  This call needs no handle and calls no cudaMalloc, cudaFree or
 * other allocating routine.  The caller passes the energy populations and a result buffer it
 * owns; the only other memory, one partial result per 256 wall nodes and a counter, is a fixed
 * array inside the library (about 160 KB, held on every GPU that loads the library until the
 * process exits).
 *
 *  lattice    lbm_lattice OR-ed with the lbm_prec of the population buffer.
 *  nx..nz     box size (nz = 1 in 2D); face_kind, T_wall and T_ref as in lbm_bc.
 *  g          device pointer to the energy populations [q_g][nz][ny][nx] in that precision's
 *             storage format: LBM_FP64 holds g itself (the layout lbm_get_populations writes),
 *             LBM_FP32 holds g - w T_ref as float, LBM_FP16S holds (g - w T_ref) * 2^10 as half
 *             (the layouts lbm_get_state writes after its 64-byte header).
 *  face       a fixed-temperature face; L and dT as in lbm_info_t.
 *  result     device pointer to 5 doubles: mean Nu, max Nu, its tangential node index, min Nu,
 *             its index (indices stored as doubles), with the definitions of lbm_nusselt.
 *  stream     cudaStream_t to run on (NULL = legacy stream); the call returns without waiting.
 * Wall temperatures are uniform per face: T_wall[f] is used at every node of face f, both in the
 * anti-bounce-back of the pulled populations and as T_w of the derivative.  A per-node profile set
 * on a handle with lbm_set_wall_profile is not seen here; for such a state use lbm_nusselt.
 * Errors: LBM_EINVAL for a bad argument, including a face with more than
 * LBM_NUSSELT_STATIC_MAX_FACE_NODES nodes (the scratch array has room for that many);
 * LBM_ECUDA if a CUDA call fails.  lbm_last_error(NULL), on the calling thread, gives the reason.
 * Set-up: the first call on each device looks up the device address of the scratch array with
 * that device current (this also creates the device's primary context if there is none yet).
 * The lookup is repeated when the device's current context has changed since, for instance after
 * cudaDeviceReset, which reloads the library's device code in a new context.  Make the first call
 * on a device, and the first call after such a reset, before any stream capture begins.  Every
 * call uses the same scratch array, which keeps the last call's contents: calls that may run at
 * the same time on the GPU (on unordered streams, or from several host threads) race and give
 * wrong results, so order them on one stream.
 */
#define LBM_NUSSELT_STATIC_MAX_FACE_NODES 1048576
LBM_API int lbm_nusselt_static(int lattice, int nx, int ny, int nz, const int face_kind[6],
                               const double T_wall[6], double T_ref, const void* g, int face,
                               double L, double dT, double* result, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Batches of 2D boxes.  The paper's studies run many independent cavities that differ in size,
 * Rayleigh and Prandtl number (Sec. 6.1: Ra = 10^3 .. 10^10 at Pr = 0.71 and grids up to 512^2;
 * Sec. 7: sweeps of Ma, resolution and Pr = 0.1 .. 5).  A batch holds such members (D2Q9 flow and
 * energy lattices, one storage precision) and advances all of them by one time step with ONE
 * kernel launch: the members' populations are concatenated in the same [q][y][x] layout, and the
 * list of every member's tiles is split into equal contiguous shares, one per block.  The grid
 * is (SM count x blocks per SM) with blocks per SM chosen by lbm_batch_set_launch or the tuner,
 * usually several times what the SMs hold at once (an oversubscribed grid), so the hardware block
 * scheduler balances the uneven members.  Each member keeps its own geometry, relaxation rates
 * and divergence flag.  Every
 * member's step is the same arithmetic as lbm_step on a handle created with the same arguments,
 * so the two give bitwise identical populations.
 * Batch handles follow the conventions of lbm_handle (allocator hook, stream, not thread-safe).
 * ------------------------------------------------------------------------------------------- */
typedef struct lbm_batch_s* lbm_batch;

typedef struct {
    int count;                      /* members */
    long long total_nodes;          /* sum of nx * ny over the members */
    int n_tiles;                    /* tiles of the current tile shape over all members */
    int tile_x, tile_y;             /* nodes per tile along x and y (one node per thread) */
    int ctas_per_sm;                /* blocks per SM of the launch (the resident count if 0 was set) */
    int grid;                       /* blocks of one step launch: min(n_tiles, SMs * ctas_per_sm) */
    int graph_steps;                /* steps per CUDA graph replay (0 = plain launches) */
    long long steps;                /* time steps taken */
    double bytes_per_node_update;   /* bytes moved per node and step (18 populations in and out) */
} lbm_batch_info_t;

/* Create a batch of `count` 2D boxes.  lattice must be LBM_D2Q9_D2Q9 OR-ed with one lbm_prec;
 * member k has size nx[k] x ny[k], Rayleigh number Ra[k], Prandtl number Pr[k], boundary and
 * initial conditions bc[k] (as lbm_create), and all members share Ma.  Every member is mapped to
 * lattice units and initialised exactly as lbm_create maps and initialises a single box.
 * Errors: LBM_ENOTSUP for a 3D lattice, LBM_EINVAL for an empty batch, a NULL array or a member
 * that lbm_create would reject (the message names the member), LBM_ENOMEM, LBM_ECUDA.
 * lbm_batch_last_error(NULL) describes a failed create. */
LBM_API int lbm_batch_create(int lattice, int count, const int* nx, const int* ny, const double* Ra,
                             const double* Pr, double Ma, const lbm_bc* bc, lbm_batch* out);
LBM_API int lbm_batch_destroy(lbm_batch b);
LBM_API int lbm_batch_set_stream(lbm_batch b, void* stream);

/* Launch shape of the step: tiles of tile_x x tile_y nodes (tile_x in {32, 64, 128, 256},
 * tile_x * tile_y <= 256 threads), ctas_per_sm blocks per SM (1..1024; 0 = as many as the SM holds
 * at once, so that every block is resident and takes one equal share of the tiles), and
 * graph_steps steps per CUDA graph replay (0..4096, rounded up to even; 0 = plain launches).
 * Default 64 x 2 tiles, ctas_per_sm 0, 32 graph steps.  Errors: LBM_EINVAL for another shape. */
LBM_API int lbm_batch_set_launch(lbm_batch b, int tile_x, int tile_y, int ctas_per_sm, int graph_steps);

/* Autotuner: time trial_steps steps of every tile shape of a fixed list, each with 1/2 to 64
 * times (at most 1024) the blocks per SM that the SM holds at once (CUDA occupancy API), on a device copy of the
 * current populations; keep the fastest and report it through the optional outputs.  The batch's own state and step count are unchanged (divergence flags are
 * cleared).  Needs device memory for two extra copies of the populations (LBM_ENOMEM otherwise). */
LBM_API int lbm_batch_tune(lbm_batch b, int trial_steps, int* tile_x, int* tile_y, int* ctas_per_sm);

/* Advance every member by n time steps (n >= 0), on the batch's stream, without waiting. */
LBM_API int lbm_batch_step(lbm_batch b, long n);

/* Wait for the batch's stream; if diverged is not NULL, diverged[k] = 1 when member k saw a
 * non-finite or non-positive density or a non-finite temperature (0 otherwise).  Returns
 * LBM_EDIVERGED if any member did. */
LBM_API int lbm_batch_sync(lbm_batch b, int* diverged);

/* Wall Nusselt numbers of a fixed-temperature face of one member, as lbm_nusselt. */
LBM_API int lbm_batch_nusselt(lbm_batch b, int member, int face, double* mean, double* nu_max,
                              double* nu_min, int* j_max, int* j_min);

/* Populations of one member as FP64 host arrays [9][ny][nx] (f and g), as lbm_get_populations
 * and lbm_set_populations. */
LBM_API int lbm_batch_get_populations(lbm_batch b, int member, double* f, double* g);
LBM_API int lbm_batch_set_populations(lbm_batch b, int member, const double* f, const double* g);

LBM_API int lbm_batch_info(lbm_batch b, lbm_batch_info_t* info);
LBM_API const char* lbm_batch_last_error(lbm_batch b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
