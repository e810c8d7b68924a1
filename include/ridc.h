/*
 * ridc.h -- C ABI of the GB300 semi-implicit RIDC library (libridc.so).
 *
 * Method: semi-implicit Revisionist Integral Deferred Correction, built from first-order
 * IMEX (forward-backward Euler) predictor and correctors (Ong, Melfi & Christlieb,
 * arXiv:1209.4297, Section III). The problem is the split initial-value problem
 *     y'(t) = f^S(t, y) + f^N(t, y),  y(a) = alpha            (Section II, eq. (ode))
 * with a linear stiff part f^S = D y, D = nu * L (centred second differences), so every
 * predictor/corrector step is one linear solve with (I - dt D)   (eq. (imex_diffusion)).
 *
 * All levels of one instance advance together in a lagged, lock-step pipeline on one GPU
 * (Section III-E): in each pipeline step every level whose inputs are ready takes one
 * step, and all their implicit solves run as one batched multi-right-hand-side solve.
 *
 * Conventions for every entry point:
 *   - Return value: RIDC_OK (0) or a negative RIDC_ERR_* code; ridc_error_string() names it.
 *     On error no output argument is written, except where stated.
 *   - Arrays are FP64, C-contiguous, row-major: [x] in 1D, [species][y][x] in 2D.
 *   - "on_device" flags say whether a pointer is a CUDA device pointer (1) or host memory (0).
 *     Host pointers may be pageable or pinned.
 *   - A handle is used by one host thread at a time. Work is ordered on the CUDA stream given
 *     at creation; calls that return data to the caller synchronise that stream.
 *   - A handle lives on the CUDA device that was current at its creation; every call on it
 *     runs there and leaves the caller's current device as it found it.
 *   - Device memory belongs to the library and is released by ridc_destroy().
 */
#ifndef RIDC_H
#define RIDC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------------------- */
#define RIDC_OK               0
#define RIDC_ERR_ARG         -1   /* invalid argument (null pointer, bad size, bad enum)   */
#define RIDC_ERR_OOM         -2   /* device or host allocation failed                      */
#define RIDC_ERR_CUDA        -3   /* a CUDA runtime call or kernel launch failed           */
#define RIDC_ERR_NONFINITE   -4   /* the solution contains NaN or Inf                       */
#define RIDC_ERR_TIMEOUT     -5   /* a bounded device-side wait gave up                     */
#define RIDC_ERR_UNSUPPORTED -6   /* valid request this build does not implement            */

/* ---- problem description ----------------------------------------------------------------- */
typedef enum {
    /* u_t + a u_x = nu u_xx on periodic [0,1), nodes x_i = i/N; f^N = -a central u_x.   */
    RIDC_ADV_DIFF_1D_PERIODIC = 0,
    /* Gray-Scott on [0,1]^2, zero-flux walls, cell centres; 2 species (u, v):
       f^N_u = -u v^2 + F (1-u), f^N_v = u v^2 - (F+k) v; D = diag(nu_u, nu_v) * L.       */
    RIDC_GRAY_SCOTT_2D_NEUMANN = 1,
    /* u_t + a u_x + b u_y = nu lap u on [0,1]^2, u = 0 on the walls, cell centres;
       f^N = -a u_x - b u_y by central differences.                                        */
    RIDC_ADV_DIFF_2D_DIRICHLET = 2,
    /* The paper's advection-diffusion example (Section IV-A): u_t + a u_x = nu u_xx on
       periodic [0,1), nodes x_i = i/N, f^N by first-order upwind differences
       (-a (u_i - u_{i-1})/h for a >= 0, -a (u_{i+1} - u_i)/h for a < 0).                */
    RIDC_ADV_DIFF_1D_UPWIND_PERIODIC = 3,
    /* The paper's viscous Burgers example (Section IV-B): u_t + (u^2/2)_x = nu u_xx on
       [0,1], u(0) = u(1) = 0; N interior nodes x_i = i/(N+1), i = 1..N; f^N from the flux
       f_{i+1/2} = (u_{i+1}^2 + u_i^2)/2: f^N_i = -(u_{i+1}^2 - u_{i-1}^2)/(4h).          */
    RIDC_BURGERS_1D_DIRICHLET = 4
} ridc_kind;

typedef enum {
    /* every step of the path in FP64 (solves by FP64 fast-diagonalisation GEMMs in 2D)     */
    RIDC_FP64 = 0,
    /* 2D solves by BF16 hi/lo split-precision GEMMs on the tensor cores (FP32 accumulation)
       plus n_refine refinement passes against the FP64 residual; right-hand sides,
       quadrature sums and solution accumulation stay FP64                                   */
    RIDC_MIXED_BF16X3 = 1,
    /* batched ensembles only: solves at FP32 accuracy on the tensor cores (FP32 operands
       split into TF32 hi + lo, three products, FP32 accumulation), right-hand sides,
       quadrature sums and solution accumulation in FP64, plus n_refine refinement passes
       against the FP64 residual                                                             */
    RIDC_FP32_SOLVE = 2,
    /* as RIDC_MIXED_BF16X3 with FP16 hi/lo operands: 22 significant bits per split instead
       of 16. A pass of either form is also limited by the tensor cores' FP32 accumulation,
       which grows with N: FP16 gains about 3x per pass at N = 256, little at N >= 1024.
       FP16's exponent range is narrow, so each operand plane is scaled by a power of two,
       2^k with max|v| 2^k in [2^(K0-1), 2^K0), K0 = 15 - ceil(log2 N), and the eigenvector
       tables by 2^(13 + floor(log2(N/2)/2)). Every intermediate of the two-sided transform
       is then at most N max|v| 2^k <= 2^15 (orthogonal transforms keep the Frobenius norm;
       the denominators are >= 1). The scale needs the plane's maximum, so the right-hand
       side and residual kernels stage FP32 values and a split kernel scales and splits them
       (one more FP32 write and read per value than the BF16 form).                           */
    RIDC_MIXED_FP16X3 = 3
} ridc_precision;

typedef enum {
    /* first-order IMEX step (forward-backward Euler), eq. (pred): RIDC-FBE, Theorem 1      */
    RIDC_PRED_FBE = 0,
    /* the third-order IMEX additive Runge-Kutta method of Section II (five stages, four
       implicit with diagonals 1/2, 2/3, 2, 1)                                              */
    RIDC_PRED_ARK3 = 1,
    /* the fourth-order IMEX additive Runge-Kutta method of Section II (seven stages, six
       implicit, every diagonal 1/2 except the last, 2/3)                                   */
    RIDC_PRED_ARK4 = 2
} ridc_predictor;

typedef struct {
    int    kind;          /* ridc_kind                                                      */
    double a, b;          /* advection velocity along x and y (unused by Gray-Scott)        */
    double F, k;          /* Gray-Scott feed and kill rates (unused otherwise)               */
    int    precision;     /* ridc_precision; 1D problems accept RIDC_FP64 only               */
    int    n_refine;      /* refinement passes of the mixed solve (0..4); ignored for FP64  */
    int    restart_every; /* restarts (Section III-E): every restart_every steps of the most
                             corrected level, all levels restart from its solution and re-enter
                             start-up; 0 = no restarts. Single integrators only (a batch
                             requires 0).                                                    */
    int    predictor;     /* ridc_predictor of level 0 (0 = RIDC-FBE). With a p0-th order ARK
                             predictor and order-1 first-order correctors the method has order
                             p0 + order - 1 (Theorem 2); corrector j then integrates with
                             p0 + j quadrature nodes (the window of Section III-C, widened),
                             and p0 + order - 1 <= 12 is required. Single integrators only (a
                             batch requires RIDC_PRED_FBE).                                  */
} ridc_problem;

/* 1D solves factor I - mu (S - 2 + S^T), mu = nu dt / h^2, into two first-order recurrences
 * run as block-wide scans. Measured against a long-double evaluation (n = 1024, one FBE step),
 * they are as accurate as an FP64 LU solve up to mu ~ 100; beyond, their relative error
 * grows about linearly with mu (1.8e-13 at mu = 1e4, 4.5e-10 at mu = 1e6, against 1.7e-14
 * and 2.0e-12 for LU), within the operator's conditioning bound (1 + 4 mu) x 2^-52
 * (tests/test_gpu_1d_stiff.py). The paper's 1D runs have mu = 0.5 to 10.                    */
typedef struct {
    int dim;              /* 1 or 2; must match the kind                                     */
    int n;                /* unknowns per side: 1D n >= 8 with (L + 1) n256 + L n + 1 <=
                             28000 doubles of shared memory, L = ceil(order / min(order, 8))
                             levels per SM and n256 = n rounded up to a multiple of 256
                             (n <= 9216 up to order 8, n <= 5551 at orders 9-12); 2D FP64
                             4 <= n <= 16384; 2D mixed: n a multiple of 256, at most 4096    */
} ridc_grid;

typedef struct ridc_ctx* ridc_handle;   /* opaque; owned by the library                      */

/* ---- lifetime ---------------------------------------------------------------------------- */

/* Create an integrator of order `order` (predictor + order-1 correctors, Theorem 1:
 * local error O(dt^{order+1})) with uniform step dt (Section III-C assumes uniform steps).
 *   nu      : diffusion coefficient per species (1 value, or 2 for Gray-Scott), > 0.
 *   order   : levels (predictor + order-1 correctors), 1 <= order <= 12 (Section III-E: 8th
 *             and 12th order stay free of the Runge phenomenon in double precision); with an
 *             ARK predictor of order p0 (problem->predictor), p0 + order - 1 <= 12.
 *   stream  : cudaStream_t used for all device work, or NULL for the legacy default stream.
 * Allocates the level-history rings and the solver tables on the current CUDA device.
 * The state is undefined until ridc_set_initial(). On error *out is untouched.            */
int ridc_create(const ridc_problem* problem, const ridc_grid* grid, const double* nu,
                double dt, int order, void* stream, ridc_handle* out);

/* Set every level to the initial data y(a) = alpha at t_0 and rewind the pipeline
 * (the start-up of Section III-E: "all nodes are initially populated with the initial
 * data at t0"). `u0` holds species*n^dim values; it is copied (stream-ordered; a host
 * source is staged through library-owned pinned memory, so the caller may reuse it on
 * return). Evaluates f^N and f of the initial state on the device.                        */
int ridc_set_initial(ridc_handle h, const double* u0, size_t count, int on_device);

/* Advance the pipeline until the most corrected level (order-1) has taken `nsteps` more
 * steps. Lower levels run ahead by at most order-1 steps and stop at the index the top
 * level's stencils need. Results do not depend on how a run is split across calls.
 * Stream-ordered; returns after launching (no synchronisation).                            */
int ridc_advance(ridc_handle h, long nsteps);

/* Copy the most corrected level eta^{order-1} at its current step into `out`
 * (species*n^dim values). Synchronises the stream; checks the copied values and returns
 * RIDC_ERR_NONFINITE (after copying) if any is NaN or Inf.                                 */
int ridc_get_solution(ridc_handle h, double* out, size_t count, int out_on_device);

/* Copy level `level`'s newest solution eta^{level}_{p} and, if step != NULL, its index p. */
int ridc_get_level(ridc_handle h, int level, double* out, size_t count, int out_on_device,
                   long* step);

/* Time t_p = p * dt of the most corrected level (t_0 = 0; p counts every step since
 * ridc_set_initial, across restarts).                                                      */
int ridc_get_time(ridc_handle h, double* t);

/* Steps taken so far by each level: steps[j] = p_j for j < nlevels (nlevels <= order),
 * counted from ridc_set_initial across restarts (after a restart every level stands at the
 * restart time).                                                                           */
int ridc_get_progress(ridc_handle h, long* steps, int nlevels);

/* ---- checkpoint / resume ---------------------------------------------------------------- */

/* Write the integrator's whole state into host memory `buf`: the steps taken by each level,
 * every slot of every level's ring (eta, f^N and, where the level keeps it, f = f^N + D eta;
 * Section III-E's memory footprint) and the problem parameters that state depends on.
 * The format is this library's own: a version-tagged header in native byte order followed
 * by FP64 values.
 *   buf == NULL : only *len is set, to the number of bytes needed.
 *   *len too small : RIDC_ERR_ARG, and *len is set to the number of bytes needed.
 * Synchronises the stream; RIDC_ERR_TIMEOUT if an earlier device-side wait gave up (the
 * state would be incomplete). A state written before ridc_set_initial is refused
 * (RIDC_ERR_ARG). On success *len is the number of bytes written.                            */
int ridc_save_state(ridc_handle h, void* buf, size_t* len);

/* Restore a state written by ridc_save_state. The handle must have been created for the
 * same problem: kind, grid, order, dt, nu, a, b, F, k and restart_every equal bit for bit
 * (precision and n_refine may differ: the state is FP64 in every precision). Continuing
 * from a loaded state gives the same numbers as continuing the saved integrator.
 * RIDC_ERR_ARG if len is short or the buffer is not a state of this problem; nothing is
 * changed then. Synchronises the stream, so `buf` may be reused on return.                 */
int ridc_load_state(ridc_handle h, const void* buf, size_t len);

/* Release all device and host memory of the handle (synchronises its stream). NULL is ok. */
void ridc_destroy(ridc_handle h);

/* Static description of a return code. Never NULL.                                         */
const char* ridc_error_string(int code);

/* ---- batched implicit solve --------------------------------------------------------------- */

/* Solve (I - dt nu_s L) delta = r for `nplanes` planes with the handle's solver (2D only):
 * plane p uses species p % species. r and delta hold nplanes*n*n values, both on the host
 * or both on the device. nplanes <= order*species. Synchronises the stream.
 * This is the batched multi-right-hand-side solve every pipeline step runs; the mixed
 * precision form includes its n_refine refinement passes.                                 */
int ridc_solve_planes(ridc_handle h, const double* r, double* delta, int nplanes,
                      int on_device);

/* Batched FP64 solve that allocates nothing. The paper has no counterpart: this entry point
 * exists for callers that cannot let a library allocate device memory -- for example a
 * simulation code that reserves all device memory for its own pool at start-up (a cudaMalloc
 * here would fail or upset its budget), or a time-critical loop that cannot afford
 * cudaMalloc/cudaFree, which may synchronise the device.
 * It computes the same (I - dt nu_s L) delta = r as ridc_solve_planes with the FP64
 * fast-diagonalisation GEMMs, without a handle:
 *   kind    : RIDC_GRAY_SCOTT_2D_NEUMANN (nu[0], nu[1]; plane p uses species p % 2) or
 *             RIDC_ADV_DIFF_2D_DIRICHLET (nu[0]).
 *   r, delta: device pointers to nplanes*n*n FP64 values, [plane][y][x]; they may alias.
 *   stream  : cudaStream_t (NULL: legacy default stream). Returns after launching.
 * Its tables and intermediates live in one fixed device array inside libridc.so (2.5 MiB,
 * held on every GPU that loads the library until the process exits). Limits: 4 <= n <= 128
 * and 1 <= nplanes <= 8; larger requests return RIDC_ERR_UNSUPPORTED. Every call rewrites
 * the whole array, so calls that overlap on the GPU (concurrent streams, other threads) race
 * and must be serialised by the caller. The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) and should therefore come before any stream capture;
 * after a cudaDeviceReset the next call looks it up again in the new context. A CUDA error
 * that an earlier, unrelated call left pending is reported as RIDC_ERR_CUDA and left in place
 * (nothing is launched). No cudaMalloc, cudaFree or other allocating routine is called.    */
int ridc_solve_planes_fixed(int kind, int n, const double* nu, double dt, const double* r,
                            double* delta, int nplanes, void* stream);

/* ---- batched ensembles ----------------------------------------------------------------------- */

/* Many independent instances of RIDC_ADV_DIFF_2D_DIRICHLET (uneven grid sides 32..512, each a
 * multiple of 32 for the parity-split solves; orders 1..4; own a, b, nu and dt) advanced
 * together by one persistent kernel launch: a cluster of CTAs integrates each instance,
 * largest instances first. Solves run at FP32 accuracy on the tensor cores (problem.precision
 * must be RIDC_FP32_SOLVE): FP32 operands split into TF32 hi + lo, three products per
 * transform (about 22 significant bits) with FP32 accumulation; everything else is FP64, as in
 * ridc_create.
 * The paper integrates one instance at a time; batching many is this library's addition.
 *   count      : number of instances; problems, grids, nu, dt, order are arrays of `count`.
 *   n_refine   : must be the same for all instances (0..4 refinement passes).
 * Device memory belongs to the library (rings per instance, per-CTA workspace).            */
typedef struct ridc_batch_ctx* ridc_batch;
int ridc_batch_create(int count, const ridc_problem* problems, const ridc_grid* grids,
                      const double* nu, const double* dt, const int* order, void* stream,
                      ridc_batch* out);

/* u0[i] points to instance i's n_i*n_i initial values (all on the host or all on the device).
 * Rewinds every instance to t_0. Synchronises the stream.                                   */
int ridc_batch_set_initial(ridc_batch b, const double* const* u0, int on_device);

/* Advance every instance until its most corrected level has taken `nsteps` more steps
 * (one kernel launch). Stream-ordered; returns after launching.                            */
int ridc_batch_advance(ridc_batch b, long nsteps);

/* Copy instance i's most corrected level (n_i*n_i values). Synchronises the stream.
 * RIDC_ERR_TIMEOUT (once) if a bounded device-side wait of an earlier advance gave up.      */
int ridc_batch_get_solution(ridc_batch b, int i, double* out, size_t count, int out_on_device);

/* Sum over instances of n_i^2: the cell-updates one top-level step performs.               */
long ridc_batch_cells(ridc_batch b);

/* Autotuner: picks the cluster size (1, 2 or 4 CTAs cooperating on each instance) and the
 * CTAs per SM (1 to 4) that run the whole batch fastest, then, at that launch shape, the
 * tile width of each grid side's tensor-core products: tiles are 128 rows by a multiple of 16
 * up to 64 half-columns that divides side/2 (narrow tiles give a cluster more tiles to share
 * on small grids, wide ones reuse each staged row more). Each trial advances `nsteps` steps
 * of the real batch. The choices are kept for later advances. Requires an initial state and
 * leaves the state undefined: call ridc_batch_set_initial afterwards.
 * *choice = CTAs per SM * 16 + cluster size; *best_ms = the fastest whole-batch trial.     */
int ridc_batch_autotune(ridc_batch b, long nsteps, int* choice, float* best_ms);

/* Tile width (half-columns per tensor-core tile) of the products for grid side `side`, or
 * RIDC_ERR_ARG if no instance of the batch has that side. Before any autotuning: the widest
 * multiple of 16 up to 64 that divides side/2.                                              */
int ridc_batch_tile_width(ridc_batch b, int side);

/* Set that tile width: a multiple of 16 up to 64 that divides side/2, else RIDC_ERR_ARG.
 * Stream-ordered after the advances already issued. Results do not depend on it.          */
int ridc_batch_set_tile_width(ridc_batch b, int side, int width);

/* Use launch shape `choice` (CTAs per SM * 16 + cluster size, as ridc_batch_autotune reports
 * it: 1 to 4 CTAs per SM, clusters of 1, 2 or 4 CTAs) for later advances, e.g. one tuned
 * earlier on the same batch. RIDC_ERR_ARG for another value.                                */
int ridc_batch_set_launch(ridc_batch b, int choice);

/* CUDA-graph launches so far: every advance (and every autotuner trial) is one graph of a
 * work-counter reset and the persistent cluster launch. -1 for NULL.                        */
long ridc_batch_graph_launches(ridc_batch b);

/* Release everything the batch holds (synchronises its stream). NULL is ok.                */
void ridc_batch_destroy(ridc_batch b);

/* ---- host-only helpers (no GPU needed) ----------------------------------------------------- */

/* The lock-step schedule of a fresh run of `nsteps` top-level steps: for each pipeline
 * step s the mask bit j of active[s] is set if level j advances in that step. Writes at
 * most `cap` entries and the number of pipeline steps to *count (RIDC_ERR_ARG if the
 * schedule is longer than cap; *count still set). 1 <= order <= 12.                        */
int ridc_schedule_plan(int order, long nsteps, unsigned* active, size_t cap, size_t* count);

/* The same plan continued from progress start[0..order) (steps taken by each level, as
 * ridc_get_progress reports them within one start) until the top level reaches nsteps:
 * what one ridc_advance call runs after earlier calls. RIDC_ERR_ARG if start is not a
 * reachable progress (negative, a level ahead of the one below, or the top past nsteps). */
int ridc_schedule_plan_from(int order, const long* start, long nsteps, unsigned* active,
                            size_t cap, size_t* count);

/* ridc_schedule_plan_from for a predictor of order p0 (ridc_predictor): level j may step from
 * n once level j-1 holds index max(n+1, p0+j-1), the last node of its p0+j-node stencil, and
 * lower levels keep p0+j+2 ring slots. start == NULL: a fresh run. With RIDC_PRED_FBE this is
 * ridc_schedule_plan_from.                                                                    */
int ridc_schedule_plan_predictor(int order, int predictor, const long* start, long nsteps,
                                 unsigned* active, size_t cap, size_t* count);

/* Quadrature weights w[j][m][i] of the corrector (Section III-C), FP64, computed exactly
 * in rational arithmetic and rounded: node i of the stencil t_b..t_{b+j}, interval
 * [t_{b+m}, t_{b+m+1}], in units of dt. Layout out[((j*order)+m)*(order)+i] for
 * 1 <= j < order, 0 <= m < j, 0 <= i <= j; other entries are set to 0.
 * `cap` must be >= order^3.                                                                 */
int ridc_quadrature_weights(int order, double* out, size_t cap);

/* ---- instrumentation ------------------------------------------------------------------------ */

#define RIDC_KERNEL_RHS       0   /* fused defect + quadrature right-hand side             */
#define RIDC_KERNEL_GEMM_TC   1   /* BF16x3 / FP16x3 tcgen05 fast-diagonalisation GEMM     */
#define RIDC_KERNEL_GEMM_F64  2   /* FP64 fast-diagonalisation GEMM                        */
#define RIDC_KERNEL_RESIDUAL  3   /* FP64 refinement residual + split                      */
#define RIDC_KERNEL_FINALIZE  4   /* solution accumulation + f^N, f of the new state       */
#define RIDC_KERNEL_1D        5   /* persistent 1D pipeline kernel                         */
#define RIDC_KERNEL_SPLIT     6   /* FP16 form: power-of-two scale + hi/lo split of staged
                                     FP32 operands                                           */
#define RIDC_KERNEL_COUNT     7

/* CUDA-event timing of kernel launches on the handle's stream: enable = 0 off, 1 every
 * launch, k > 1 only the launches of every k-th 2D pipeline step (steps 0, k, 2k, ...
 * counted from ridc_set_initial), which keeps the events' own cost small. Any call clears
 * the counters; enable < 0 is RIDC_ERR_ARG.                                                 */
int ridc_set_profiling(ridc_handle h, int enable);

/* Launch count and summed device time (ms) of one kernel kind since profiling was enabled.
 * Synchronises the stream.                                                                  */
int ridc_get_kernel_stats(ridc_handle h, int kernel, long* launches, double* total_ms);

/* Kernel launches issued so far by the handle (all kinds, counted on the host).            */
long ridc_launch_count(ridc_handle h);

/* ---- device memory ------------------------------------------------------------------------ */

/* Route the library's device allocations through the caller's allocator (for example a
 * framework's caching pool) instead of cudaMalloc / cudaFree.
 *   alloc(bytes, device, ctx): a device pointer to at least `bytes` bytes on `device` (the
 *     handle's device, current during the call), aligned to 256 bytes, or NULL when out of
 *     memory. The call that needed the memory then returns RIDC_ERR_OOM and gives back what
 *     it had allocated. A pointer that is not 256-byte aligned is handed back to free and
 *     the call returns RIDC_ERR_CUDA.
 *   free(ptr, bytes, device, ctx): takes back a pointer alloc returned, with its size. The
 *     library synchronises the stream (or, with no stream, the device) that used the memory
 *     before it calls free, so the memory is idle when it is returned.
 * Both NULL: cudaMalloc / cudaFree again (the default). Process-wide. RIDC_ERR_ARG when only
 * one of the two is given, or while any handle or batch exists (every buffer is freed by
 * the allocator that made it). Host staging memory (pinned) is not affected.              */
typedef void* (*ridc_alloc_fn)(size_t bytes, int device, void* ctx);
typedef void (*ridc_free_fn)(void* ptr, size_t bytes, int device, void* ctx);
int ridc_set_allocator(ridc_alloc_fn alloc, ridc_free_fn free_fn, void* ctx);

/* ---- test hooks: failures made on purpose, for the error paths ---------------------------- */

/* Make the k-th device allocation from now on (k >= 1) fail as if the device were out of
 * memory; 0 disarms. Process-wide. Every entry point that allocates then returns
 * RIDC_ERR_OOM and releases what it had allocated. RIDC_ERR_ARG for k < 0.                */
int ridc_debug_fail_alloc(int k);

/* Make the next tensor-core GEMM launch of the handle leave one operand stage unloaded, so
 * that the barrier its consumer waits on never completes. Every device-side wait is bounded
 * (2 s of %globaltimer): the launch gives up, flags the handle's error and frees its tensor
 * memory, and the next call that synchronises (ridc_solve_planes, ridc_get_solution, ...)
 * returns RIDC_ERR_TIMEOUT and clears the flag. The context stays usable. Mixed-precision
 * 2D handles only (RIDC_ERR_UNSUPPORTED otherwise).                                         */
int ridc_debug_stall_next_gemm(ridc_handle h);

#ifdef __cplusplus
}
#endif

#endif /* RIDC_H */
