/*
 * selm_mg.h - C ABI of the GB300 stochastic multigrid library for the
 * Stochastic Eulerian-Lagrangian Method (Atzberger, "Spatially Adaptive
 * Stochastic Multigrid Methods for Fluid-Structure Systems with Thermal
 * Fluctuations", arXiv:1003.2680).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every pointer argument named as a field, particle array or output is a
 *   DEVICE pointer owned by the caller, unless stated otherwise.  The library
 *   never frees caller memory.
 * - Every call is enqueued on `stream` (a cudaStream_t passed as void*; NULL =
 *   the legacy default stream) and returns before the GPU work finishes,
 *   except where a host-visible result (cycle counts, residuals) is asked
 *   for, which synchronises `stream`.
 * - Argument errors are reported synchronously as a status code; no C++
 *   exception crosses the ABI.  The text of the last error of a handle is
 *   returned by selm_mg_last_error().
 * - Geometry: the unit box [0,1]^d, periodic in x (and y in 3-D), no-slip
 *   walls at z = 0 and z = 1 (in 2-D the paper's y axis is called z here).
 *   n cells per axis, h = 1/n.  Velocity components live on the MAC faces
 *   normal to their axis (Section 4); the wall-normal component has n-1
 *   unknowns along z (its wall nodes are Dirichlet 0), the others n.
 * - Field layout: a "field" of a system at a level is the concatenation of
 *   its components, each a row-major array [nz][ny][nx] (x fastest, ny = 1 in
 *   2-D).  selm_mg_layout() returns every size and offset.  Particle arrays
 *   X, F, U, g are row-major [np][dim] doubles; in 2-D the columns are (x, z).
 * - Operator: A = mu h^d (-L_h), the SPD scaled MAC Laplacian (Section 2.1,
 *   Eq. equ_H_selm_discr with alpha = h^-d absorbed), so that the mobility is
 *   M = Gamma P~ A^-1 P~ Gamma^T and the thermal field is
 *   g = sqrt(2 kT) Gamma P~ xi with xi ~ N(0, A^-1) (Eqs. equ_G_special_form,
 *   equ_g_gen_xi).
 */
#ifndef SELM_MG_H
#define SELM_MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct selm_mg selm_mg;  /* opaque handle, owned by the library */

typedef enum {
  SELM_OK = 0,
  SELM_EINVAL = 1,   /* malformed descriptor or argument */
  SELM_ENOMEM = 2,   /* device allocation failed */
  SELM_ECUDA = 3,    /* a CUDA call failed (text in selm_mg_last_error) */
  SELM_ENOCONV = 4,  /* FAC solve did not reach tol within max_cycles */
  SELM_ETIMEOUT = 5, /* a bounded device-side wait ran out */
  SELM_EBUSY = 6     /* no free slot / memory for admission */
} selm_status;

enum { SELM_FP64 = 0, SELM_FP32_REFINE64 = 1 };          /* precision */
enum { SELM_PROJ_NONE = 0, SELM_PROJ_MAC = 1 };           /* projection */
enum { SELM_COARSE_CHOLESKY = 0, SELM_COARSE_SMOOTH = 1 }; /* coarsest level */
enum { SELM_SYS_VELOCITY = 0, SELM_SYS_PRESSURE = 1 };    /* system selector */

typedef struct {
  int dim;                 /* 2 or 3 */
  int n;                   /* cells per axis; divisible by 2^(levels-1) */
  double mu;               /* viscosity (Eq. equ_fld_cont) */
  double kT;               /* thermal energy k_B T (Eq. equ_effective_fluct) */
  int levels;              /* multigrid levels; 0 = coarsen while the edge stays even and >= 4 */
  int nu_pre, nu_post;     /* (mu1, mu2) smoothing sweeps of Algorithm 3; 0 -> 2 */
  int precision;           /* SELM_FP64 or SELM_FP32_REFINE64 */
  int projection;          /* SELM_PROJ_NONE (P~ = I) or SELM_PROJ_MAC */
  int coarse_mode;         /* SELM_COARSE_CHOLESKY (exact block step) or SELM_COARSE_SMOOTH (Alg. 3 literally) */
  double tol;              /* FAC stop: ||b - Az||_2 <= tol ||b||_2 ; 0 -> 1e-10 */
  int max_cycles;          /* FAC cycle cap; 0 -> 100 */
  double proj_tol;         /* pressure-solve tolerance of the projection; 0 -> 1e-10 */
  int max_particles;       /* capacity of the particle scratch of selm_mg_step; 0 -> 4096 */
  uint64_t seed;           /* Philox key material (noise of this chain) */
  uint64_t instance;       /* Philox key material (distinguishes systems) */
  /* optional device allocator hooks (e.g. a framework's caching allocator);
     NULL -> cudaMalloc / cudaFree.  The returned memory must be 256-byte
     aligned (the kernels use vector accesses); create fails with
     SELM_EINVAL otherwise. */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
} selm_mg_desc;

/* Device bytes a handle for `desc` will allocate (state + scratch); 0 if the
   descriptor is invalid.  Used for admission by footprint. */
size_t selm_mg_footprint(const selm_mg_desc* desc);

/* Validate `desc`, build the Galerkin hierarchy on the host (Section 3.2,
   A^(l) = P^T A^(l-1) P with trilinear P), factor the coarsest operators,
   allocate and upload device state on `stream`.  *out receives the handle. */
selm_status selm_mg_create(const selm_mg_desc* desc, void* stream, selm_mg** out);
selm_status selm_mg_destroy(selm_mg* h);
const char* selm_mg_last_error(const selm_mg* h);

/* ---- the SELM operations (Algorithm 4) ---------------------------------- */

/* U = M F = Gamma P~ A^-1 P~ Gamma^T F (Alg. 4 step 2): spread, project,
   FAC-solve to tol (Algorithm 1), project, interpolate.  Each projection's
   pressure solve starts from the pressure of the same projection in the
   previous call (Algorithm 1 takes an initial value); selm_mg_project alone
   starts from zero.  X, F: [np][dim]
   positions and forces; U: [np][dim] output.  cycles_out / resid_out are
   optional HOST pointers (synchronises the stream when given). */
selm_status selm_mg_solve(selm_mg* h, int np, const double* X, const double* F, double* U,
                          int* cycles_out, double* resid_out, void* stream);

/* Advance the persistent chain xi by `ncycles` stochastic FAC cycles
   (Alg. 4 step 3, b = 0) and return g = sqrt(2 kT) Gamma P~ xi at X.
   xi_out (optional, device) receives a copy of xi (velocity field layout). */
selm_status selm_mg_sample(selm_mg* h, int np, const double* X, int ncycles, double* g,
                           double* xi_out, void* stream);

/* `nsteps` Euler-Maruyama steps (Alg. 4 steps 1-5) with fixed forces F:
   X <- X + Gamma P~ (dt A^-1 P~ Gamma^T F + sqrt(2 kT dt) xi), then periodic
   wrap and reflection at the walls.  X is updated in place.  With the
   projection, each step's chain cycles run on a stream of the handle beside
   the solve, and the solve runs on a high-priority stream of the handle;
   both fork from `stream` and join back to it before the call returns, so
   work later enqueued on `stream` sees the whole step. */
selm_status selm_mg_step(selm_mg* h, int np, double* X, const double* F, double dt, int nsteps,
                         int ncycles_per_step, void* stream);

/* selm_mg_step on HOST arrays: copies X and F (row-major [np][dim] doubles in
   host memory, ideally pinned) to the device, runs `nsteps` steps, copies X
   back and synchronises `stream`.  np <= max_particles. */
selm_status selm_mg_step_host(selm_mg* h, int np, double* X_host, const double* F_host, double dt,
                              int nsteps, int ncycles_per_step, void* stream);

/* ---- layout and state --------------------------------------------------- */

int selm_mg_levels(const selm_mg* h, int system);
int selm_mg_ncomp(const selm_mg* h, int system);
/* dims3 = {nx, ny, nz} of component `comp` at `level`; *offset = its element
   offset in the level field; *level_size = elements of the whole field. */
selm_status selm_mg_layout(const selm_mg* h, int system, int level, int comp, int* dims3,
                           long long* offset, long long* level_size);
/* Element size (4 or 8) of the inner (level) fields of the handle. */
int selm_mg_inner_bytes(const selm_mg* h);
/* Device pointer of the chain state xi (velocity layout, FP64) and its cycle
   counter (the Philox counter of the next stochastic cycle). */
selm_status selm_mg_chain(selm_mg* h, double** xi, uint64_t* cycle);
/* Device pointer of the velocity field u of the handle's current FAC solve
   (velocity layout, FP64, owned by the handle): after a step, the solution of
   A u = Gamma^T F of its last velocity solve (Alg. 4 step 2); with
   SELM_PROJ_MAC the right-hand side is the projected spread force. */
selm_status selm_mg_velocity(selm_mg* h, double** u);
selm_status selm_mg_set_cycle(selm_mg* h, uint64_t cycle);
/* Failure-path hook: raises the timeout flag of `system`'s cooperative waits
   (on `stream`), as a wait that ran out of time does.  The next cooperative
   level launch gives up at its first wait and returns; the next norm read of
   a solve reports SELM_ECUDA and clears the flag.  Lets a test exercise the
   failure path without a GPU fault. */
selm_status selm_mg_fail_waits(selm_mg* h, int system, void* stream);
/* Options.  SELM_OPT_COARSE_ENGINE (default 1): run the levels below the
   finest with the cluster-resident coarse engine (one thread-block cluster
   per component, colour passes separated by cluster barriers); 0 selects one
   launch per colour pass.  Both give the same result up to rounding. */
enum {
  SELM_OPT_COARSE_ENGINE = 1,
  SELM_OPT_ENGINE_CLUSTER = 2,
  SELM_OPT_ENGINE_LEVEL = 3,
  SELM_OPT_LEVEL_COOP = 4,
  SELM_OPT_GRAPHS = 5,
  SELM_OPT_SPECULATE = 6,
  SELM_OPT_PRESSURE_SPECTRAL = 8
};
/* SELM_OPT_ENGINE_CLUSTER: largest thread-block cluster the coarse engine may
   use (1..16; 0 = the largest that fits).  Re-plans the engine; synchronises
   the legacy default stream.
   SELM_OPT_ENGINE_LEVEL: first level the coarse engine may take (0 = the
   first level whose slabs fit in shared memory); the levels above it run as
   GPU-wide launches.  Re-plans both systems' engines.
   SELM_OPT_LEVEL_COOP (default 1): each half V-cycle of a level above the
   engine runs as one cooperative launch over every SM.  1: with FP32 inner
   cycles the colour passes run in dataflow order, each site update waiting
   for its coupled neighbours only (each stored value carries the parity of
   its update count in its least significant mantissa bit, at most 1 ulp from
   the rounded update); FP64 levels, and levels whose stencil admits no such
   order, separate the passes by grid barriers.  2: grid barriers always.
   Every wait is bounded; a timed-out wait is reported as SELM_ECUDA by the
   next solve's norm read.  0 selects one launch per colour pass.  All give
   the same result up to rounding. */
/* SELM_OPT_GRAPHS (default 1): the V-cycles of solves and chain cycles on the
   handle's own buffers are captured once as CUDA graphs (on a stream of the
   handle) and replayed, which removes their per-launch host cost and launch
   gaps; same launches and results.  0 launches every kernel directly (for
   short-lived handles, where capture would not pay off).
   SELM_OPT_SPECULATE (default 1): while a solve's previous residual and
   contraction predict no convergence, its next V-cycle is enqueued before the
   residual norm is read back (the correction is applied only if the norm
   confirms: same iterates and cycle counts), so the device does not idle
   during the read-back; 0 waits for every norm first (for handles that share
   the GPU with other work, where a mispredicted V-cycle costs others).
   SELM_OPT_PRESSURE_SPECTRAL (default 1 where available): the projection's
   pressure problem (D^ D^T) phi = D^ w (Section 4) keeps its FP64 iterative
   refinement (Algorithm 1) but takes the exact inner solve of the uniform
   channel's Neumann operator -- FFT along x and y, a tridiagonal solve along z
   per mode, FFT back, in FP32 -- instead of the pressure system's V-cycle;
   available for FP32 inner cycles on 3-D grids with nx == ny a power of two
   up to 128 (SELM_EINVAL elsewhere).  0 selects the V-cycle.  Both stop at
   proj_tol.
   Setting any option on a handle that holds captured graphs synchronises the
   device and drops them. */
selm_status selm_mg_set_option(selm_mg* h, int option, int value);
/* 1 when the handle's projections use the spectral inner solve (their
   pressure "cycles" in selm_mg_stats are then refinement iterations, not
   V-cycles), else 0. */
int selm_mg_pressure_spectral(const selm_mg* h);
/* Coarse engine of `system`: first level it covers (-1 = not used), cluster
   size and dynamic shared memory per CTA. */
selm_status selm_mg_engine_info(const selm_mg* h, int system, int* first_level, int* cluster_size,
                                size_t* smem_bytes);
/* FAC cycles run by the last solve (velocity) and the projections it did. */
selm_status selm_mg_stats(const selm_mg* h, int* last_solve_cycles, int* last_proj_cycles,
                          long long* total_vcycles);

/* ---- method steps on caller buffers (one entry per hot-path step) -------
   v, b, d, r: inner-precision fields (selm_mg_inner_bytes) of `system` at
   `level` in the layout above.  z, b64: FP64 level-0 fields.  `cycle` is the
   Philox counter; noise != 0 draws the Gaussian terms (sampling),
   noise == 0 runs the deterministic smoother (solving). */

/* Section 3.1 / Alg. 3 steps 1,5: one full stochastic Gauss-Seidel sweep,
   z_i <- (b_i - sum_{j!=i} A_ij z_j)/A_ii + n_i/sqrt(A_ii), red-black at
   level 0 and multicolour on the Galerkin levels; `sweep` is the index
   within the cycle (0..mu1-1 pre, mu1.. post) used in the noise counter. */
selm_status selm_mg_smooth(selm_mg* h, int system, int level, void* v, const void* b, int sweep,
                           uint64_t cycle, int noise, void* stream);
/* Alg. 3 step 3: b_coarse = P^T (b - A^(level) v) for level -> level+1. */
selm_status selm_mg_residual_restrict(selm_mg* h, int system, int level, const void* v,
                                      const void* b, void* b_coarse, void* stream);
/* Alg. 3 step 4: v += P v_coarse (level+1 -> level). */
selm_status selm_mg_prolong_correct(selm_mg* h, int system, int level, void* v,
                                    const void* v_coarse, void* stream);
/* Coarsest level (reading of Alg. 3 step 2): v = A_c^-1 b + noise * L_c^-T n,
   A_c = L_c L_c^T in FP64 (exact block heat-bath). */
selm_status selm_mg_coarsest(selm_mg* h, int system, void* v, const void* b, uint64_t cycle,
                             int noise, void* stream);
/* Alg. 3 V-cycle on the correction equation at level 0: v <- V-Cycle(v, b). */
selm_status selm_mg_vcycle(selm_mg* h, int system, void* v, const void* b, uint64_t cycle,
                           int noise, void* stream);
/* Alg. 1 step 1 in FP64: r = b64 - A z (b64 may be NULL = 0), stored in the
   inner precision; if norm2 (device double) is given, adds ||r||^2 to it. */
selm_status selm_mg_outer_residual(selm_mg* h, int system, const double* z, const double* b64,
                                   void* r, double* norm2, void* stream);
/* Alg. 1 step 4 in FP64: z += d. */
selm_status selm_mg_outer_update(selm_mg* h, int system, double* z, const void* d, void* stream);
/* One FAC iteration (Algorithm 1) on FP64 z: z <- z + V-Cycle(0, b - A z). */
selm_status selm_mg_fac_cycle(selm_mg* h, int system, double* z, const double* b64, uint64_t cycle,
                              int noise, void* stream);
/* Deterministic FAC iteration from the given z until ||b - Az|| <= tol ||b||
   (synchronises to read the norm). */
selm_status selm_mg_fac_solve(selm_mg* h, int system, double* z, const double* b64, double tol,
                              int max_cycles, int* cycles_out, double* resid_out, void* stream);
/* Section 2.1 coupling: b = Gamma^T F (Peskin 4-point spreading onto the
   velocity unknowns; b is overwritten). */
selm_status selm_mg_spread(selm_mg* h, int np, const double* X, const double* F, double* b,
                           void* stream);
/* U = Gamma u (Peskin 4-point interpolation of the velocity field u). */
selm_status selm_mg_interp(selm_mg* h, int np, const double* X, const double* u, double* U,
                           void* stream);
/* Section 4 / Section 2.1: w <- P~ w = w - D^T (D D^T)^+ D w, the MAC
   projection, by a deterministic FAC solve of the Neumann pressure problem. */
selm_status selm_mg_project(selm_mg* h, double* w, int* cycles_out, void* stream);
/* Alg. 4 step 4 tail: X += V, wrap the periodic coordinates, reflect at walls. */
selm_status selm_mg_em_update(selm_mg* h, int np, double* X, const double* V, void* stream);

/* One V-cycle like selm_mg_vcycle (velocity system) for callers that cannot
   allocate device memory: no cudaMalloc, no pinned host buffer, no allocator
   hook.  Such callers are, for example, a service that plans its whole device
   memory budget up front and forbids allocation once it runs, or a thread
   that cannot reach the allocator of the framework that owns the device.
   The paper has no counterpart; this is a deployment convenience.
   Its scratch (Galerkin tables, coarse-level fields, the level-0 residual
   buffer, counters, the coarse-engine plan) lives in one fixed 16 MiB device
   array that every device loading this library keeps until the process
   exits; grids whose scratch does not fit (3-D: roughly above 80^3 in FP32,
   64^3 in FP64) are rejected with SELM_EINVAL and a message on stderr.
   `desc` describes the grid as for selm_mg_create (projection and allocator
   fields are ignored); v and b are level-0 inner-precision fields in the
   selm_mg_layout order.  The first call on a device, and the first call
   after the descriptor changes, builds the hierarchy into the array: it
   looks up the array's device address, copies the tables and synchronises
   `stream`, so make that call before any stream capture (a set-up requested
   on a capturing stream is refused with SELM_EINVAL).  All calls share the
   array: the level fields are cleared inside each V-cycle and the counter
   slot is rewritten per call, but calls that overlap on the GPU (other
   streams, other threads) race.  Host calls from several threads are
   serialised per device. */
selm_status selm_mg_vcycle_static(const selm_mg_desc* desc, void* v, const void* b, uint64_t cycle,
                                  int noise, void* stream);

/* ---- batched form ---------------------------------------------------------
   Many independent systems (uneven sizes, own seeds and kT) advanced
   together.  Each phase of a step (spread + initial residual; one V-cycle of
   every solve; the stochastic chain cycles; combine + interpolate + move) is a
   CUDA graph with one branch per system, captured on the first call with a
   given set of particle arrays and dt, and replayed afterwards; the FAC solve
   (Algorithm 1) takes one graph launch per V-cycle for all systems and stops
   when every system meets its tolerance (systems that met it earlier take
   the extra cycles).  Systems must use SELM_PROJ_NONE.  Profiling
   (selm_profile_enable) must be off while graphs are captured. */
typedef struct selm_batch selm_batch;
selm_status selm_batch_create(int nsys, const selm_mg_desc* descs, void* stream, selm_batch** out);
selm_status selm_batch_destroy(selm_batch* b);
/* Handle of system i (for layouts, chain state, statistics); owned by the batch. */
selm_mg* selm_batch_system(selm_batch* b, int i);
const char* selm_batch_last_error(const selm_batch* b);
/* nsteps Euler-Maruyama steps for every system: np[i], X[i] (device,
   [np][dim], updated in place), F[i]; solve_cycles (optional host [nsys])
   receives the FAC cycles each system needed in the last step. */
selm_status selm_batch_step(selm_batch* b, const int* np, double* const* X, const double* const* F, double dt,
                            int nsteps, int ncycles_per_step, int* solve_cycles, void* stream);
/* Autotuner: times one FAC cycle of every system for each tile shape of the
   persistent form (see selm_batch_set_persistent) and for engine cluster sizes
   16, 8 and 4 of the graph form, keeps the best shape of each and runs the
   faster form from then on (selm_batch_info tells which); *chosen_cluster
   receives the graph form's cluster size. */
selm_status selm_batch_autotune(selm_batch* b, int* chosen_cluster, void* stream);
enum { SELM_BATCH_SOLVE = 0, SELM_BATCH_SAMPLE = 1 };
/* One FAC cycle (Algorithm 1) of every system of the batch, the systems side
   by side on the batch's branch streams, joined into `stream`:
   SELM_BATCH_SAMPLE: one stochastic cycle of each system's thermal chain
     (b = 0, noise on); the chain counters advance by one;
   SELM_BATCH_SOLVE: one deterministic cycle of each system's velocity solve
     from its current iterate u (selm_mg_velocity) and right-hand side (those
     of its last step): u <- u + V-Cycle(0, b - A u).
   Other modes return SELM_EINVAL. */
selm_status selm_batch_cycle(selm_batch* b, int mode, void* stream);
/* Persistent form (the default when every system has the same inner
   precision and sweep counts, the exact coarsest step and level-0 rows of
   8-wide segments, until selm_batch_autotune finds the graph form faster):
   every FAC cycle of all systems
   (Algorithm 1 around Algorithm 3) is one cooperative launch that walks the
   cycle's phases -- FP64 residual, each colour pass of each level, residual and
   restriction, the coarsest exact step, prolongation, FP64 update -- for every
   system, aligned by level, with a grid barrier between phases and each
   system's own noise counters, so every system's result is what it computes
   alone.  selm_batch_step captures the solve cycle (with the residual norms'
   read-back) and the chain cycles as CUDA graphs; its tile shapes (z rows per
   level-0 column item: 8, 16, 32; co-resident blocks per SM: 1, 2) come from
   selm_batch_autotune.  on = 0 selects the
   per-system graphs (SELM_EINVAL if the batch does not qualify for on = 1).
   Synchronises the device. */
selm_status selm_batch_set_persistent(selm_batch* b, int on);
/* Form and tile shape of the batch: persistent (0/1), z rows per level-0
   column item, blocks per SM, engine cluster size of the graph form. */
selm_status selm_batch_info(const selm_batch* b, int* persistent, int* kc, int* blocks_per_sm, int* cluster);
/* Profiling aid of the persistent form: runs one FAC cycle of every system
   (mode as selm_batch_cycle; SELM_BATCH_SOLVE runs the cycle from u) with a
   %globaltimer stamp after each phase and returns, per phase, its type (0
   FP64 residual, 1 colour pass, 2-3 the coarsest step's two triangular
   solves, 4 residual, 5 restriction, 6 prolongation, 7 FP64 update), its
   level and its duration in microseconds (types/levels/us: host arrays of
   max_phases entries; *nphases receives the count; SELM_EINVAL when it
   exceeds max_phases).  Synchronises `stream`. */
selm_status selm_batch_phase_times(selm_batch* b, int mode, int max_phases, int* types, int* levels, double* us,
                                   int* nphases, void* stream);

/* ---- served form -----------------------------------------------------------
   A request loop.  One device pool of `budget_bytes` is reserved at creation;
   requests are admitted in arrival order as soon as a contiguous block of
   their footprint (selm_mg_footprint of the request's descriptor) is free in
   the pool and one of `max_slots` worker threads is idle.  Each admitted
   request keeps its system on the device, runs selm_mg_step_host on its own
   stream (copy X and F in, nsteps steps, copy X out) and releases its block;
   the admitted requests' work overlaps on the GPU.  X and F are HOST arrays
   that must stay valid until the request's result has been polled; X is
   overwritten with the final positions.  The descriptor's allocator hooks are
   ignored (the pool serves the workspace). */
typedef struct {
  selm_mg_desc desc;     /* the system of this request (grid, walls, kT, seeds) */
  int np;                /* particles */
  double* X;             /* host [np][dim], updated in place */
  const double* F;       /* host [np][dim] */
  double dt;
  int nsteps;
  int ncycles_per_step;
  void* user;            /* returned with the result */
} selm_request;

typedef struct {
  uint64_t id;
  void* user;
  selm_status status;
  double t_submit, t_admit, t_done;   /* seconds on the server clock */
  int vcycles;                        /* V-cycles the request ran */
} selm_result;

typedef struct selm_server selm_server;
selm_status selm_server_create(size_t budget_bytes, int max_slots, selm_server** out);
/* Continuous batching (the served form on the batched engine): one
   scheduler keeps up to `max_slots` admitted requests resident and runs the
   next Euler-Maruyama step of all of them as one batched step
   (selm_batch_step over the requests' handles: per-phase graph launches
   shared by all, or with `persistent` the persistent batched FAC launch, one
   work-list slot per request, where the systems qualify).  Between steps the
   requests whose nsteps are done are copied out and retired, waiting
   requests are admitted (arrival order, footprint in the pool, the running
   batch's dt and chain cycles per step; an empty batch takes the next
   request's), and the batch is rebuilt over the new membership.  Requests
   must be SELM_PROJ_NONE systems (submit returns SELM_EINVAL otherwise).
   Each request's result equals its run alone up to the extra FAC cycles a
   batched solve gives the systems that converge first. */
selm_status selm_server_create_batched(size_t budget_bytes, int max_slots, int persistent, selm_server** out);
/* Batched steps run and batch rebuilds (membership changes) so far. */
selm_status selm_server_batch_stats(selm_server* s, long long* steps, long long* rebuilds);
/* Queues a request (returns at once); SELM_EBUSY if it can never fit the pool. */
selm_status selm_server_submit(selm_server* s, const selm_request* r, uint64_t* id);
/* Moves up to `max` finished results to `out`; returns how many. */
int selm_server_poll(selm_server* s, selm_result* out, int max);
/* Waits until every submitted request has finished. */
selm_status selm_server_drain(selm_server* s);
/* Peak pool bytes and busy slots since creation, current bytes and queue length. */
selm_status selm_server_stats(selm_server* s, size_t* peak_bytes, int* peak_slots, size_t* bytes_in_use,
                              int* queued);
/* Seconds since the server was created (the clock of selm_result). */
double selm_server_clock(selm_server* s);
/* Finishes the queued requests, stops the workers and frees the pool. */
selm_status selm_server_destroy(selm_server* s);

/* ---- exact discrete Stokes mobility and the Ito drift ---------------------
   Corrections beyond the paper's effective dynamics (which uses
   M = Gamma P~ A^-1 P~ Gamma^T and drops kT div_X M, Section 2.1).
   selm_mg_stokes_solve: u = S f, the velocity of the MAC saddle point
   A u + D^T p = f, D u = 0 (D the integer MAC divergence), by conjugate
   gradients on the pressure Schur complement D A^-1 D^T with FAC inner solves
   (Algorithm 1) a hundred times tighter than `tol` (0: the descriptor's tol);
   f, u: device velocity fields (level-0 layout).  iters / resid (optional
   HOST) receive the outer iterations and the relative Schur residual; the
   call synchronises.  The first Stokes call allocates the handle's Stokes
   scratch (through the descriptor's allocator hooks if given).
   selm_mg_stokes_mobility: U = Gamma S Gamma^T F.
   selm_mg_rfd_directions: W ([np][dim], device) of step `step`: Philox
   kind 3 normals, rank = particle * dim + axis, counter words 2-3 = step.
   selm_mg_rfd_drift: d = (kT / delta) [M_S(X + delta W/2) - M_S(X - delta W/2)] W,
   the random finite difference of kT div_X M_S.
   selm_mg_stokes_step: `nsteps` Euler-Maruyama steps with both corrections:
   d at the start positions (W of the handle's step counter, which advances
   by one per step; delta = 0 omits the drift), the chain advanced by
   `ncycles`, then X <- X + Gamma S (dt Gamma^T F + sqrt(2 kT dt) A xi) + dt d,
   wrapped and reflected.  Independent of the descriptor's projection. */
selm_status selm_mg_stokes_solve(selm_mg* h, const double* f, double* u, double tol, int* iters, double* resid,
                                 void* stream);
selm_status selm_mg_stokes_mobility(selm_mg* h, int np, const double* X, const double* F, double* U, void* stream);
selm_status selm_mg_rfd_directions(selm_mg* h, int np, uint64_t step, double* W, void* stream);
selm_status selm_mg_rfd_drift(selm_mg* h, int np, const double* X, const double* W, double delta, double* d,
                              void* stream);
selm_status selm_mg_stokes_step(selm_mg* h, int np, double* X, const double* F, double dt, int nsteps, int ncycles,
                                double delta, void* stream);

/* ---- measurement --------------------------------------------------------
   Process-wide kernel accounting.  selm_kernel_launches() counts every
   kernel this library has launched since it was loaded.  With profiling on,
   every launch is bracketed by CUDA events recorded on its own stream;
   selm_profile_read() synchronises on those events and returns, per kernel
   class, the summed device time (ms) and the number of launches since the
   last reset.  Do not enable profiling while a stream is being captured. */
enum {
  SELM_K_FINE_SWEEP = 0,    /* red-black colour pass, level 0 */
  SELM_K_COARSE_SWEEP = 1,  /* multicolour pass, Galerkin levels */
  SELM_K_RESIDUAL = 2,
  SELM_K_RESTRICT = 3,
  SELM_K_PROLONG = 4,
  SELM_K_COARSEST = 5,
  SELM_K_OUTER_RESIDUAL = 6,
  SELM_K_OUTER_UPDATE = 7,
  SELM_K_SPREAD = 8,
  SELM_K_INTERP = 9,
  SELM_K_PROJECTION = 10,
  SELM_K_OTHER = 11,
  SELM_K_BATCH_CYCLE = 12,  /* persistent batched FAC cycle (all systems, one launch) */
  SELM_K_NCLASSES = 13
};
long long selm_kernel_launches(void);
selm_status selm_profile_enable(int on);
selm_status selm_profile_reset(void);
selm_status selm_profile_read(int kernel_class, double* total_ms, long long* launches);

/* Philox4x32-10 (Salmon et al., SC'11) of n counters: ctr and out are device
   arrays of 4n uint32.  A utility for checking the noise generator. */
selm_status selm_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, uint32_t* out,
                               int n, void* stream);

/* ===================================================================== *
 * Composite grid with one refined patch: FAC of Algorithms 1 and 2.
 *
 * The base channel (dim 2 or 3; n cells along each periodic axis; wall axis
 * with its cell centres on the walls, unknown rows j = 1..n-1, Section 4's
 * Dirichlet rule) has its rows j = 1..K next to the bottom wall refined by 2
 * over the whole x-y extent.  Each of `ncomp` scalar components is a
 * cell-centred field; the operator is Section 4's adaptive discretization
 * L = DG (Eqs. equ_def_discr_div to equ_def_L: face-area-weighted divergence,
 * the 3/4-spacing gradient across coarse-fine faces with the coarse face
 * carrying the mean of its fine faces), used in the symmetric form
 * A = -mu V L.  One FAC iteration (Algorithm 1 around Algorithm 2):
 * r = b - A z (FP64); the residual restricted to the base grid (the transpose
 * of the parent-copy prolongation); one V-cycle (Algorithm 3) on the Galerkin
 * base hierarchy; the correction copied into the patch; nu_patch Gibbs sweeps
 * of the patch cells with the composite rows (four passes per sweep: red,
 * then the red interface-layer cells with odd x, then the same for black);
 * z += correction.  Noise of the patch sweeps: Philox counter kind 2; the
 * four cells of one colour in an 8-cell x segment of a patch row share a
 * block: group = row * ceil(2n / 8) + x / 8 (row = layer * rows_per_layer +
 * y), lane = (x mod 8) / 2.
 *
 * Composite vectors are FP64 device arrays of selm_comp_size() elements: the
 * patch (per component [2K][2n][2n], 2-D [2K][1][2n], x fastest) followed by
 * the base grid (per component [n-1][n][n], 2-D [n-1][1][n]).  The base rows
 * j <= K are covered by the patch and are not unknowns: they are ignored on
 * input, left unchanged in z and zero in residual outputs.
 * ===================================================================== */
typedef struct selm_comp selm_comp;

typedef struct {
  int dim;          /* 2 or 3 */
  int n;            /* base cells per periodic axis: even, >= 4 */
  int K;            /* refined base rows next to the bottom wall: 1 <= K <= n-2 */
  int ncomp;        /* scalar components 1..3 (0 = 1); component ids 0..ncomp-1 */
  int levels;       /* base multigrid levels (0 = coarsen while the edge stays even and >= 4) */
  int nu_pre, nu_post, nu_patch;   /* Algorithm 2/3 sweep counts (0 = 2) */
  int precision;    /* SELM_FP64 or SELM_FP32_REFINE64 (inner cycles FP32, FP64 residual) */
  int coarse_mode;  /* SELM_COARSE_CHOLESKY or SELM_COARSE_SMOOTH */
  double mu;        /* viscosity (0 = 1) */
  uint64_t seed, instance;   /* Philox key material, as for selm_mg_desc */
  void* (*alloc)(size_t bytes, void* ctx);   /* optional workspace hooks (NULL: cudaMalloc) */
  void (*free)(void* p, void* ctx);
  void* alloc_ctx;
} selm_comp_desc;

/* Device bytes a handle needs (0 for an invalid descriptor). */
size_t selm_comp_footprint(const selm_comp_desc* desc);
/* Creates the handle (synchronises `stream`).  SELM_EINVAL: invalid
   descriptor; SELM_ENOMEM: no workspace. */
selm_status selm_comp_create(const selm_comp_desc* desc, void* stream, selm_comp** out);
selm_status selm_comp_destroy(selm_comp* c);
const char* selm_comp_last_error(const selm_comp* c);
/* Elements of a composite vector. */
long long selm_comp_size(const selm_comp* c);
/* Layout of part 0 (patch) or 1 (base grid) of component `comp` in a
   composite vector: dims (x, y, z) and element offset. */
selm_status selm_comp_layout(const selm_comp* c, int part, int comp, int dims[3], long long* offset, long long* size);
/* Bytes of the inner (level-field) precision: 4 or 8. */
int selm_comp_inner_bytes(const selm_comp* c);
/* r = b - A z on the composite unknowns (FP64; b may be NULL for 0; covered
   rows of r are 0); *norm2 (optional, host) receives ||r||^2.  Synchronises
   `stream` when norm2 is given. */
selm_status selm_comp_residual(selm_comp* c, const double* z, const double* b, double* r, double* norm2,
                               void* stream);
/* `count` Gibbs sweeps of the patch cells of A q = r, with inner-precision
   level fields: q_patch (patch field, updated), q_base (base field, read:
   the coarse neighbours of the top layer), r_patch (patch field).  Counter
   cycle `cycle`; noise 0 = plain Gauss-Seidel. */
selm_status selm_comp_patch_sweeps(selm_comp* c, void* q_patch, const void* q_base, const void* r_patch, int count,
                                   uint64_t cycle, int noise, void* stream);
/* One FAC iteration on z (b may be NULL for 0) with Philox cycle `cycle`. */
selm_status selm_comp_fac_cycle(selm_comp* c, double* z, const double* b, uint64_t cycle, int noise, void* stream);
/* Deterministic FAC iterations from the value in z until ||b - A z|| <=
   tol ||b|| (SELM_ENOCONV after max_cycles).  Synchronises `stream`. */
selm_status selm_comp_solve(selm_comp* c, double* z, const double* b, double tol, int max_cycles, int* cycles,
                            double* rel, void* stream);
/* Advances the handle's chain xi ~ N(0, A^-1) by `ncycles` stochastic FAC
   iterations (b = 0; counter cycle = chain step); copies the state into
   xi_out (an FP64 composite vector, optional) on `stream`.  With FP32 inner
   cycles the chain is kept as a double-float pair (hi + lo, about 48
   significant bits) whose residual and update run on the FP32 pipes; with
   SELM_FP64 it is an FP64 vector. */
selm_status selm_comp_sample(selm_comp* c, int ncycles, double* xi_out, void* stream);
/* Cycle counter of the next chain step. */
selm_status selm_comp_chain(selm_comp* c, uint64_t* cycle);
selm_status selm_comp_set_cycle(selm_comp* c, uint64_t cycle);
/* FAC iterations run by the handle. */
selm_status selm_comp_stats(const selm_comp* c, long long* total_cycles);

#ifdef __cplusplus
}
#endif
#endif /* SELM_MG_H */
