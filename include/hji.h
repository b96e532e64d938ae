/*
 * hji.h - C ABI of the GB300 (sm_103a) solver for warm-start Hamilton-Jacobi-
 * Isaacs reachability (Herbert, Ghosh, Bansal, Tomlin, arXiv:1903.07715).
 *
 * The library time-marches the infinite-horizon avoid HJI variational
 * inequality of Sec. II-B, Eq. (7),
 *     min{ D_t V + H(x, grad V), l(x) - V } = 0,
 * backwards in time on a dense N-D grid (N <= 4), with the Hamiltonian of
 * Eq. (6), H = max_u min_d <grad V, f(x,u,d)>, for control-affine dynamics
 * (Eq. (1)) with box-bounded control and disturbance.  It starts from the
 * standard initialisation V(x,0) = l(x) (Sec. II-B) or from a warm start
 * V(x,0) = min(k(x), l(x)) (Sec. III, Eq. (14) and the proof of Thm. 1), and
 * stops when the largest change of V over the grid in one step falls below a
 * tolerance (Sec. IV), or at a horizon / step cap.
 *
 * Numerics (the paper delegates them to a level-set toolbox, Sec. II-B after
 * Eq. (8)): upwind one-sided derivatives (ENO1, ENO2, HJ-WENO5), the
 * Lax-Friedrichs numerical Hamiltonian with dissipation coefficients
 * alpha_a = max over the grid of max_{u,d} |f_a|, TVD Runge-Kutta of order
 * 1/2/3 with dt = cfl / max over the grid of sum_a max_{u,d}|f_a| / dx_a, and
 * V <- min(V, l) after every full step.  Ghost nodes beyond a non-periodic
 * edge extrapolate V linearly from the two edge nodes.
 *
 * Conventions for every entry point:
 *   - Arrays are dense, C order (axis 0 slowest), element type double for
 *     HJI_F64 grids and float for HJI_F32 grids.
 *   - Node i of axis a sits at lo[a] + i * dx[a], dx[a] = (hi[a]-lo[a])/(n[a]-1),
 *     or (hi[a]-lo[a])/n[a] on a periodic axis.
 *   - `ptr_is_device` = 1: the pointer is CUDA device memory on the current
 *     device; 0: host memory.  The library never keeps caller pointers beyond
 *     a call; every call that reads or writes caller memory has finished with
 *     it when it returns.
 *   - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).
 *     All device work of a call is ordered on it; calls return after that
 *     work has finished.
 *   - No exception or C++ object crosses this boundary.  Errors are returned
 *     as hji_status; hji_last_error() gives a per-handle message.
 *   - A handle is not thread-safe; separate handles may be used from
 *     separate threads.
 */
#ifndef HJI_H
#define HJI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HJI_MAX_DIM 4    /* state dimensions per grid            */
#define HJI_MAX_INPUTS 4 /* control / disturbance components     */
#define HJI_MAX_TERMS 8  /* nonlinear terms w * phi(x[axis])     */

typedef struct hji_grid_s* hji_grid;

typedef enum {
    HJI_OK = 0,
    HJI_E_INVALID = 1,       /* bad argument, NaN/Inf input, unsupported size          */
    HJI_E_NOMEM = 2,         /* device allocation failed                               */
    HJI_E_CUDA = 3,          /* a CUDA runtime call failed (see hji_last_error)        */
    HJI_E_NOT_CONVERGED = 4, /* horizon or step cap reached first; value still valid   */
    HJI_E_TIMEOUT = 5,       /* a bounded device wait gave up                          */
    HJI_E_STATE = 6,         /* call out of order (no dynamics set, no value yet, ...) */
    HJI_E_NONFINITE = 7,     /* the march produced NaN/Inf (e.g. cfl too large)         */
    HJI_E_CHECK = 8          /* bounds-checked debug build only: an index check of the
                                tile/halo code failed (hji_last_error names the site,
                                the index and the extent); the access was redirected
                                to element 0, so the value is not meaningful          */
} hji_status;

typedef enum { HJI_F64 = 0, HJI_F32 = 1 } hji_precision;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns device memory of `bytes` bytes usable on `stream` (NULL on
 * failure); free releases it.  NULL allocator: cudaMallocAsync/cudaFreeAsync. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, void* stream, void* ctx);
    void* ctx;
} hji_allocator;

/* Create a grid of ndim (1..4) axes with n[a] >= 3 nodes on [lo[a], hi[a]]
 * (hi > lo), at most 2^31 - 1 nodes in all, periodic[a] != 0 for a periodic
 * axis (may be NULL), storing V in `prec`.  The grid is the discretised
 * state space on which Sec. II-B computes the value function (the standard
 * initialisation there sets V = l at every grid state; the update of each
 * grid state after Eq. (8) is the march of hji_solve); node placement and
 * spacing are stated at the top of this header.  Allocates the value
 * buffers on the current device.  `alloc` may be NULL; if not, it is copied and must
 * stay callable until hji_grid_destroy.
 * Errors: HJI_E_INVALID (sizes, bounds), HJI_E_NOMEM, HJI_E_CUDA. */
hji_status hji_grid_create(int ndim, const int64_t* n, const double* lo, const double* hi,
                           const int* periodic, hji_precision prec, const hji_allocator* alloc,
                           hji_grid* out);

/* Release every device buffer of the grid.  NULL is accepted.  The paper
 * has no counterpart (resource management of this C ABI). */
hji_status hji_grid_destroy(hji_grid g);

typedef enum { HJI_FN_TAN = 0, HJI_FN_SIN = 1, HJI_FN_COS = 2 } hji_fn;

/* Control-affine dynamics of Sec. II-A, Eq. (1), with n = the grid's ndim:
 *   f(x,u,d) = c + A x + sum_t term_w[t] * phi_t(x[term_axis[t]]) e_{term_row[t]}
 *              + G u + E d,
 *   u in [ulo, uhi] (m components), d in [dlo, dhi] (q components).
 * Layouts (row-major, dense): c[n], A[n*n] (A[i*n+j] multiplies x_j in f_i),
 * G[n*m], E[n*q]; term arrays of length nterms, phi given as hji_fn.
 * m in 0..4, q in 0..4, nterms in 0..8; c, A, E, term arrays may be NULL when
 * unused (zero).  Requires ulo <= uhi and dlo <= dhi componentwise, all
 * values finite.  The arrays are copied; the caller keeps ownership.
 * Errors: HJI_E_INVALID. */
typedef struct {
    int m, q, nterms;
    const double* c;
    const double* A;
    const double* G;
    const double* E;
    const int* term_row;
    const int* term_axis;
    const int* term_fn;
    const double* term_w;
    const double* ulo;
    const double* uhi;
    const double* dlo;
    const double* dhi;
} hji_dynamics;

hji_status hji_dynamics_set(hji_grid g, const hji_dynamics* dyn);

typedef enum { HJI_ENO1 = 1, HJI_ENO2 = 2, HJI_WENO5 = 5 } hji_scheme;

typedef enum {
    HJI_INIT_STANDARD = 0, /* V(x,0) = l(x)                                        */
    HJI_INIT_USER_K = 1,   /* V(x,0) = min(k(x), l(x)), k given by the caller      */
    HJI_INIT_RESIDENT = 2  /* V(x,0) = min(V_prev(x), l(x)): the grid's last value */
} hji_init;

/* scheme: ENO1 (needs n >= 3), ENO2 (n >= 5), WENO5 (n >= 7) per axis.
 * rk_order: 1, 2 or 3.  cfl in (0, 1].  tol >= 0: stop once max|dV| < tol.
 * horizon >= 0: stop once tau >= horizon (0 = none).  max_steps: step cap
 * (<= 0 means 1,000,000).  check_every: steps per host check of the stop
 * flag (<= 0 means 32); steps after the stop point never run.  Results do
 * not depend on check_every or the tile shape (see march below). */
typedef struct {
    hji_scheme scheme;
    int rk_order;
    double cfl;
    double tol;
    double horizon;
    int check_every;
    int64_t max_steps;
    hji_init init;
    int tile_variant; /* 0: the autotuned (else default) tile shape;
                         1..HJI_TILE_VARIANTS: force shape tile_variant-1 (2-D) */
    double tol_rate;  /* >= 0: the test becomes max|dV| < tol + tol_rate * dt, a
                         bound on the rate of change; tol = 0, tol_rate = 0.1 is
                         Sec. IV's rule (change < 0.001 per 0.01 of time) */
    int march;        /* how the steps are launched (results are identical):
                         HJI_MARCH_AUTO, HJI_MARCH_PER_STAGE or
                         HJI_MARCH_MULTI_STEP */
    double interval;  /* > 0: also stop once the largest change of V over one
                         interval of this much time is below interval_tol:
                         Sec. V's test (interval 0.01, interval_tol 0.001).
                         An interval is K = max(1, round(interval / dt)) CFL
                         steps; V is compared with its copy from K steps
                         earlier after every K-th step.  0: off. */
    double interval_tol; /* >= 0, see interval */
    int brs;          /* 0: the VI of Eq. (7), V <- min(V, l) after every step
                         (the tube, the default); 1: the HJI PDE of Eq. (5)
                         alone, no projection onto V <= l: the value of the
                         backward reachable set at time tau (normally run to
                         a horizon); a warm start k (or the resident value)
                         is then taken as it is, not as min(k, l) */
    int local_lf;     /* 0: Lax-Friedrichs dissipation with the grid-wide
                         alpha_a (default); 1: with the node's own
                         alpha_a(x) = max_{u,d} |f_a(x,u,d)| (dt stays the
                         grid-wide CFL step).  Local dissipation marches with
                         one launch per stage and the default tile shape. */
    double discount;  /* 0 (or 1): off.  gamma in (0, 1): discounted
                         reachability (Sec. II-C): each step ends with
                         V <- min(l, gamma * V~), V~ the Runge-Kutta step's
                         result, instead of min(l, V~); gamma = exp(-lambda dt)
                         is the factor of one CFL step.  The map is then a
                         contraction, so any start converges, to a value with
                         the same sign as the undiscounted one.  Sec. V's
                         schedule (0.999, then 1 once converged) is two
                         calls: a discounted solve, then an undiscounted one
                         from the resident value.  Not with brs. */
} hji_solve_opts;

/* hji_solve_opts.march.  PER_STAGE: one kernel launch per Runge-Kutta
 * stage, check_every steps captured in one CUDA graph.  MULTI_STEP: one
 * cooperative launch runs every stage of check_every steps, with a
 * bounded grid-wide barrier after each stage (no launch gaps, no per-launch
 * ramp and tail); it exists for 1-D and 2-D grids (3-D/4-D ones would
 * spill registers) and needs every CTA resident at once: elsewhere it falls
 * back to PER_STAGE.  AUTO: MULTI_STEP for 1-D and 2-D grids whose stages
 * give every resident CTA at least 4 tiles (the barrier then costs less
 * than a kernel boundary), PER_STAGE otherwise.  Both forms run the same per-node arithmetic from the same
 * source; compiled as different kernels, the compiler may fuse a different
 * set of multiply-adds, so their results agree to rounding, not bit for bit.
 * Within one form, results do not depend on check_every, on the batch an
 * instance marches in, or on the tile shape. */
#define HJI_MARCH_AUTO 0
#define HJI_MARCH_PER_STAGE 1
#define HJI_MARCH_MULTI_STEP 2

typedef struct {
    int64_t steps;       /* full Runge-Kutta steps taken                      */
    double tau;          /* backward time reached (steps * dt)                */
    double dt;           /* CFL step used                                     */
    double final_max_dV; /* max |V^{n+1} - V^n| of the last step (FP64)       */
    double wall_ms;      /* host wall time of the call                        */
    double alpha[HJI_MAX_DIM]; /* Lax-Friedrichs coefficients                 */
    int converged;       /* 1 if final_max_dV < tol ended the march           */
    int64_t kernel_launches; /* device kernels this call launched (set-up,
                                stages, and the no-op stages queued past the
                                stop point)                                   */
} hji_solve_stats;

/* March the HJI VI (Sec. II-B, Eq. (7); min(., l) after every full step,
 * Eq. (8)) on grid g for target l (grid-shaped) from the init mode in `o`
 * (V0 = l, Sec. II-B, or the warm start V0 = min(k, l), Sec. III); k is
 * read only for HJI_INIT_USER_K (else may be NULL).  The result stays in
 * the grid (read it with hji_value_get; HJI_INIT_RESIDENT starts
 * the next solve from it).  Returns HJI_OK when converged,
 * HJI_E_NOT_CONVERGED when a cap stopped it first (the value is still the
 * last iterate), HJI_E_INVALID for bad options or NaN/Inf in l or k,
 * HJI_E_STATE if no dynamics were set (or RESIDENT without a prior value),
 * HJI_E_NONFINITE if the march blew up, HJI_E_NOMEM / HJI_E_CUDA.
 * `stats` may be NULL. */
hji_status hji_solve(hji_grid g, const void* l, const void* k, int ptr_is_device,
                     const hji_solve_opts* o, void* cuda_stream, hji_solve_stats* stats);

/* Several grids in one march (each grid is the march of Sec. II-B, Eq. (7),
 * exactly as hji_solve runs it; the paper solves one problem at a time and
 * has no batched form): every RK stage of every grid is one persistent
 * kernel launch over a shared tile list, captured in CUDA graphs; each grid
 * stops on its own test while the others go on.  All grids must share
 * precision and ndim; l[i], k[i] belong to grids[i] (k may be NULL, or hold
 * NULL entries, unless o->init is HJI_INIT_USER_K).  stats has `count`
 * entries or is NULL.  Returns HJI_OK if every grid converged, else the
 * first non-OK per-grid status. */
hji_status hji_batch_solve(int count, hji_grid* grids, const void* const* l,
                           const void* const* k, int ptr_is_device, const hji_solve_opts* o,
                           void* cuda_stream, hji_solve_stats* stats);

/* Copy the grid's current value (grid-shaped, the grid's precision) to out:
 * the value function V(x, tau) of Sec. II-B, Eq. (4), at the nodes, which
 * after a converged solve is the infinite-horizon value V*(x) of Eq. (7)
 * whose sub-zero level set is the unsafe set (Sec. II-B, after Eq. (5)).
 * Errors: HJI_E_STATE (no value yet), HJI_E_INVALID, HJI_E_CUDA. */
hji_status hji_value_get(hji_grid g, void* out, int ptr_is_device, void* cuda_stream);

/* Allocation-free one-shot solve.  The paper has no counterpart: this entry
 * serves callers that may not allocate device memory themselves (code whose
 * device memory is owned by a host framework, real-time loops that forbid
 * allocator calls, processes whose allocator is exhausted).  The caller
 * passes device pointers: l (input), k (input, read for HJI_INIT_USER_K;
 * NULL otherwise) and v_out (output, grid-shaped, the grid's precision; for
 * HJI_INIT_RESIDENT it also holds the previous value on entry).  Grid,
 * dynamics and options mean what they mean for hji_grid_create,
 * hji_dynamics_set and hji_solve, with these differences: tile_variant 0
 * takes the default tile shape (no autotuned choice is consulted); the
 * march always launches one kernel per RK stage (opts.march is ignored);
 * the interval test needs a snapshot buffer and is refused (opts.interval
 * != 0 returns HJI_E_INVALID); and an FP32 HJI_INIT_RESIDENT start begins
 * from the float values in v_out alone, while hji_solve's resident FP32
 * start also carries the low words of its compensated value, so the two
 * marches may differ by FP32 rounding.
 * Every scratch buffer lives in one static
 * device array of HJI_NOALLOC_SCRATCH_BYTES bytes that each GPU loading the
 * library holds until exit; a grid that needs more (5 values per node for
 * FP64 RK3, 7 for FP32 RK3, rows padded to a multiple of 8 nodes, plus small
 * tables) returns HJI_E_INVALID.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, once per device and CUDA context: a call in a new
 * context of the device, e.g. after cudaDeviceReset, looks it up again);
 * make it before any stream capture (a look-up due inside a capture is
 * refused with HJI_E_STATE).  Calls share the array: calls whose GPU work overlaps race.  No
 * cudaMalloc, cudaFree or other allocating routine is called.  Errors as for
 * hji_solve; the message is in hji_noalloc_last_error(). */
#define HJI_NOALLOC_SCRATCH_BYTES (32u << 20)
hji_status hji_solve_noalloc(int ndim, const int64_t* n, const double* lo, const double* hi,
                             const int* periodic, hji_precision prec, const hji_dynamics* dyn,
                             const void* l, const void* k, void* v_out,
                             const hji_solve_opts* o, void* cuda_stream, hji_solve_stats* stats);
/* The message of this thread's last failed hji_solve_noalloc call.  The
 * paper has no counterpart (error reporting of this C ABI). */
const char* hji_noalloc_last_error(void);

/* Copy src's current value into dst as dst's resident value (converting
 * precision on the device), so that hji_solve(dst, ..., HJI_INIT_RESIDENT)
 * starts from it.  This is how an FP32 march is followed by an FP64
 * re-validation sweep warm-started from its result (by Thm. 1 / Thm. 2 that
 * sweep is conservative, and exact when the FP32 value lies above the FP64
 * solution).  Grids must have the same ndim and node counts.  An FP32 source
 * contributes its full compensated value (high + low word); an FP64 source
 * is split exactly into an FP32 high and low word.
 * Errors: HJI_E_INVALID (shape), HJI_E_STATE (src has no value), HJI_E_CUDA. */
hji_status hji_value_transfer(hji_grid dst, hji_grid src, void* cuda_stream);

/* ---- Continuous-batching engine (serving) ----
 * One engine marches many requests at once: each request is a grid (its
 * dynamics already set with hji_dynamics_set), a target l and an init mode
 * (typically HJI_INIT_RESIDENT: warm-start from the solution the grid kept
 * from its previous request, Sec. III).  Requests wait in a queue and are
 * admitted into slots while others are marching, as long as a slot is free
 * and the device bytes of the admitted grids stay within the budget; every
 * chunk of check_every steps advances all admitted requests with one
 * persistent kernel launch per RK stage (a CUDA graph that reads the
 * device-side tile list, so admissions and departures need no re-capture);
 * a request leaves when its own test stops it and its slot refills at the
 * next step.  A request's arithmetic does not depend on what else is in the
 * batch, so its result equals a solo hji_solve bit for bit.
 * All grids of an engine share ndim and precision; the options (scheme,
 * rk_order, cfl, tol, tol_rate, interval, interval_tol, horizon, max_steps,
 * check_every) are the engine's.  Engines always launch one kernel per RK
 * stage (opts.march is ignored), so that engines on different streams
 * interleave on the device.
 * hji_engine_step never blocks on the chunk it launches: it waits for the
 * previous chunk, retires and admits, then launches the next, so engines on
 * different streams overlap on the device when stepped in turn. */
typedef struct hji_engine_s* hji_engine;

/* max_slots: 1..65535 concurrent requests; budget_bytes: device bytes the
 * admitted grids may hold together (0 = no limit).  alloc (may be NULL:
 * cudaMallocAsync) supplies the engine's own device buffers (descriptors,
 * counters, tile list); it is copied and must stay callable until
 * hji_engine_destroy.  Errors: HJI_E_INVALID, HJI_E_NOMEM, HJI_E_CUDA. */
hji_status hji_engine_create(int ndim, hji_precision prec, const hji_solve_opts* o, int max_slots,
                             size_t budget_bytes, void* cuda_stream, const hji_allocator* alloc,
                             hji_engine* out);

/* Queue a request.  l (grid-shaped, host or device) is copied into the grid
 * now, on the engine's stream; k likewise for HJI_INIT_USER_K.  A grid may
 * have one request queued or marching at a time (HJI_E_STATE otherwise), and
 * must not be used outside the engine until that request is polled.  A
 * grid larger than the whole budget is refused with HJI_E_INVALID. */
hji_status hji_engine_submit(hji_engine e, hji_grid g, const void* l, const void* k,
                             int ptr_is_device, hji_init init, int64_t tag);

/* Wait for the chunk in flight, retire finished requests, admit queued ones,
 * launch the next chunk.  *active / *queued (may be NULL) report the slots
 * in use and the requests waiting after the call. */
hji_status hji_engine_step(hji_engine e, int* active, int* queued);

/* Finished requests since the last poll: up to `cap` of (tag, stats,
 * status); *count receives how many were written. */
hji_status hji_engine_poll(hji_engine e, int64_t* tags, hji_solve_stats* stats,
                           hji_status* status, int cap, int* count);

/* Release the engine (requests still queued or marching are dropped).  The
 * paper has no counterpart (resource management of this C ABI). */
hji_status hji_engine_destroy(hji_engine e);
/* The message of the engine's last failed call.  The paper has no
 * counterpart (error reporting of this C ABI). */
const char* hji_engine_last_error(hji_engine e);

/* Tile-shape autotuner (the paper has no counterpart).  2-D grids can be
 * marched with HJI_TILE_VARIANTS tile shapes (31x32, 15x64 and 63x16 nodes,
 * rows x columns); this times `steps` steps of a
 * standard march of grid g (dynamics set, target l) with each (one warm-up
 * march, then the median of three timed ones) and remembers
 * the fastest for this precision, ndim, scheme, RK order and grid-size class
 * (log2 of the node count).  Later hji_solve, hji_batch_solve and engines
 * of that class use it (the nearest tuned size class; untuned: variant 0).
 * The timing march overwrites g's value.  chosen (may be NULL) receives the
 * variant; ms_per_step (may be NULL, HJI_TILE_VARIANTS entries) the wall
 * time per step of each variant (-1 where not applicable).  Grids of other
 * dimensionality have one shape (chosen = 0). */
#define HJI_TILE_VARIANTS 3
hji_status hji_autotune(hji_grid g, const void* l, int ptr_is_device, const hji_solve_opts* o,
                        int steps, void* cuda_stream, int* chosen, double* ms_per_step);

/* Per-stage kernel durations (the paper has no counterpart; a measurement aid
 * for the stage kernels of the time march of Sec. II-B).  Runs `steps` (1..4096)
 * steps of the march from V0 = l with o's scheme, RK order, CFL and tile
 * shape (o's tol, horizon, max_steps, check_every and init are ignored),
 * launching each RK stage kernel on its own between two CUDA events on
 * cuda_stream instead of inside a graph, and writes the mean duration in
 * milliseconds of RK stage i's kernel to ms_per_stage[i] (rk_order entries,
 * caller-owned; entry rk_order-1 is the last stage, fused with min(., l) of
 * Eq. (7)-(8) and the max|dV| reduction).  The kernels are those of
 * hji_solve, so the grid's value afterwards equals that of hji_solve with
 * tol = 0 and max_steps = steps.  Synchronous.  Errors: as hji_solve, and
 * HJI_E_INVALID for steps out of range or ms_per_stage NULL. */
hji_status hji_stage_times(hji_grid g, const void* l, int ptr_is_device, const hji_solve_opts* o,
                           int steps, void* cuda_stream, double* ms_per_stage);

/* Self-test of the bounded waits inside the stage kernels (the paper has no
 * counterpart).  Every wait of a stage kernel on a TMA copy gives up after a
 * time limit and the kernel records HJI_E_TIMEOUT for the instance, instead
 * of hanging the GPU.  This call runs the same wait routine on one CTA whose
 * mbarrier is armed for bytes that no copy delivers, with limit_ns
 * (1e6 .. 4e9 nanoseconds), and returns HJI_E_TIMEOUT when the wait gave up
 * (the expected result), HJI_E_STATE if the barrier completed, HJI_E_INVALID
 * for a limit out of range, HJI_E_NOMEM / HJI_E_CUDA on runtime failures.
 * Synchronous on cuda_stream; the message is in hji_last_error(NULL). */
hji_status hji_selftest_bounded_wait(int64_t limit_ns, void* cuda_stream);

/* Which build this library is, and a self-test of its index-check recorder
 * (the paper has no counterpart).  The library also comes as a
 * bounds-checked debug build (_hji_checked.so, the same sources compiled
 * with HJI_CHECKED): there every index the stage kernels' tile and halo code
 * forms is tested against its array's extent before the access; a failed
 * check is recorded for the instance, the access goes to element 0 instead,
 * and the solve returns HJI_E_CHECK with the first failure in
 * hji_last_error.  *checked (may be NULL) is 1 in that build, 0 in the
 * product build.  The self-test runs the recorder on fixed indices that are
 * compared, never used as addresses (one inside a 10-element extent, a
 * 4-wide range past its end, one before its start, a failed condition) and
 * returns how many failures it recorded (*count: 3 in the checked build, 0
 * in the product build, whose checks compile to nothing) and the first one
 * (*site, *index, *extent; may be NULL).  Synchronous on cuda_stream.
 * Errors: HJI_E_NOMEM, HJI_E_CUDA (message in hji_last_error(NULL)), and
 * HJI_E_STATE if the recorder returned other indices than it should. */
hji_status hji_selftest_index_check(void* cuda_stream, int* checked, int* count, int* site,
                                    int64_t* index, int64_t* extent);

/* The instantaneous optimal control of Sec. II-B, Eq. (9),
 *     u*(x) = argmax_u min_d <grad V(x), f(x,u,d)>,
 * at every node of the grid's current value (normally a converged V*), and
 * the disturbance d*(x) attaining the inner minimum.  grad V is the average
 * (p- + p+)/2 of `scheme`'s one-sided derivatives (the gradient at which the
 * march evaluates the Hamiltonian, same ghost nodes).  Over the boxes the
 * choice separates by component: u*_j = uhi_j where (G^T grad V)_j >= 0, else
 * ulo_j; d*_k = dlo_k where (E^T grad V)_k >= 0, else dhi_k (a zero
 * component, where every value is optimal, takes uhi_j / dlo_k).  Computed
 * in the grid's precision (FP32 grids: from the compensated value).
 * u_out: m grid-shaped dense arrays one after another (u_out[j*N + node],
 * N nodes, C order, the grid's precision); d_out: q such arrays, or NULL.
 * Synchronous.  Errors: HJI_E_INVALID (NULL grid or u_out with m > 0,
 * scheme, grid too small for the stencil), HJI_E_STATE (no dynamics or no
 * value yet), HJI_E_NOMEM, HJI_E_CUDA. */
hji_status hji_optimal_control(hji_grid g, hji_scheme scheme, void* u_out, void* d_out,
                               int ptr_is_device, void* cuda_stream);

/* Measured fused-multiply-add rate of the current GPU in `prec` (a
 * measurement aid for the arithmetic roofline of the stage kernels; the
 * paper has no counterpart).  Every thread of a grid that fills every SM
 * runs independent multiply-add chains; the loop count is calibrated so a
 * launch takes about target_ms (1 .. 1000), five launches are timed with
 * CUDA events on cuda_stream, and the fastest gives *tflops (one FMA = two
 * floating-point operations) and *ms_per_launch (may be NULL).  Allocates
 * nothing; synchronous.  Errors: HJI_E_INVALID (precision, target_ms,
 * tflops NULL), HJI_E_CUDA; the message is in hji_peak_last_error(). */
hji_status hji_peak_fma(hji_precision prec, double target_ms, void* cuda_stream, double* tflops,
                        double* ms_per_launch);
/* The message of this thread's last failed hji_peak_fma call.  The paper
 * has no counterpart (error reporting of this C ABI). */
const char* hji_peak_last_error(void);

/* Grid facts: ndim, n[], and the number of nodes (may be NULL each).  The
 * paper has no counterpart (introspection of this C ABI). */
hji_status hji_grid_info(hji_grid g, int* ndim, int64_t* n, int64_t* num_nodes);

/* Static text of a status code ("unknown status" for other values).  The
 * paper has no counterpart: error reporting of this C ABI only. */
const char* hji_status_string(hji_status s);
/* The paper has no counterpart: error reporting of this C ABI only.
 * The message of the last failed call on grid g; for g NULL, of the last
 * failed call on this thread that had no grid (hji_grid_create, NULL
 * arguments, hji_selftest_bounded_wait).  Owned by the library, valid until
 * the next call that fails the same way. */
const char* hji_last_error(hji_grid g);

#ifdef __cplusplus
}
#endif
#endif /* HJI_H */
