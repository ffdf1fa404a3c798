/*
 * mgrit.h -- C ABI of the GB300 (sm_103a) MGRIT library for method-of-lines
 * discretisations of 1D periodic linear advection (De Sterck, Falgout,
 * Krzysik, Schroder, arXiv 2209.06916).
 *
 * Problem (Sec. 2.1, Eq. ad and Eq. one-step-general): u_t + alpha u_x = 0 on
 * [-1, 1) with periodic boundaries, nx equispaced points x_i = -1 + i h
 * (h = 2/nx), nt steps of size dt, CFL number c = alpha dt / h (Sec. 4.3).
 * The fine one-step map is Phi = R_q(-c L_p) (Eq. MOL_M_def): order-p upwind
 * finite differences L_p (Sec. 4.1) with an ERKq or SDIRKq method (Sec. 4.2).
 * Coarse level l >= 1 uses the corrected semi-Lagrangian operator
 * Phi^{(m^l dt)} = (I - phi_l D^{(p+1)}_2)^{-1} S_p^{(m^l dt)} (Eq.
 * MOL-SL-corrected and its multilevel form with the phi recursion, Sec. 6.2).
 * MGRIT itself is the linear two-level / V-cycle method of Sec. 2.2 with
 * F(CF)^nu pre-relaxation and F post-relaxation.
 *
 * Conventions for every entry point
 *  - Return value: MGRIT_OK (0) or a negative MGRIT_ERR_* code; the text of a
 *    code is mgrit_strerror(code).  No entry point aborts the process.
 *  - Pointers marked "host or device" may point to host memory or to device
 *    memory of the handle's GPU; the kind is detected with
 *    cudaPointerGetAttributes.  "device" pointers must be device memory.
 *  - Vectors are FP64, row-major: index [k * nx + i] for time row k and grid
 *    index i.  The caller owns every pointer it passes; the handle owns every
 *    buffer it allocates (freed by mgrit_destroy).
 *  - All GPU work of a handle is issued on the stream given to mgrit_setup
 *    (0 = the legacy default stream).  Entry points that return host results
 *    synchronise that stream before returning.
 *  - A handle is not thread safe; distinct handles are independent.
 */
#ifndef MGRIT_H_
#define MGRIT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define MGRIT_OK 0
#define MGRIT_ERR_INVALID_ARG -1   /* bad size / parameter / pointer            */
#define MGRIT_ERR_OOM -2           /* device allocation failed or over budget   */
#define MGRIT_ERR_NOT_CONVERGED -3 /* max_iter reached; stats are filled        */
#define MGRIT_ERR_DIVERGED -4      /* residual non-finite or growing 1e3-fold    */
#define MGRIT_ERR_TIMEOUT -5       /* a bounded device-side wait gave up        */
#define MGRIT_ERR_CUDA -6          /* a CUDA runtime call failed                */
#define MGRIT_ERR_UNSTABLE -7      /* a coarse correction matrix is singular or */
                                   /* has an unstable factorisation             */
#define MGRIT_ERR_UNSUPPORTED -8   /* valid parameters this build cannot run    */

/* ---- enumerations ------------------------------------------------------ */
#define MGRIT_ERK 0   /* explicit RK, stability polynomial R_q (Sec. 4.2)      */
#define MGRIT_SDIRK 1 /* singly diagonally implicit RK (Sec. 4.2)              */

#define MGRIT_FP64 0  /* every kernel in FP64                                  */
#define MGRIT_MIXED 1 /* FP32 relaxation sweeps inside FP64 iterative          */
                      /* refinement: FP64 C-point residual and norm (level 0),*/
                      /* FP64 coarsest sequential solve and FP64 truncation-  */
                      /* error correction solves                              */
#define MGRIT_MIXED_FAST 2 /* as MGRIT_MIXED, but the correction solves run  */
                      /* in FP32 on levels whose correction matrix has        */
                      /* condition number <= 1e6 (FP64 on the others; the     */
                      /* environment variable MGRIT_FAST_KAPPA sets the bound) */

#define MGRIT_MAX_LEVELS 16
#define MGRIT_COARSE_SL_CORRECTED 0
#define MGRIT_COARSE_SL 1
#define MGRIT_COARSE_REDISC 2
#define MGRIT_SOLVE_DIRECT 0 /* exact periodic banded correction solve        */
#define MGRIT_SOLVE_GMRES 1  /* GMRES correction solve (Sec. 6.1, Sec. 6.3)   */
#define MGRIT_MAX_HISTORY 128

/* ---- parameters -------------------------------------------------------- */
typedef struct mgrit_params {
  int64_t nx;       /* grid points, 32 <= nx, nx % 8 == 0                       */
  int64_t nt;       /* time steps; nt % (m m_coarse^(levels-2)) == 0            */
  double cfl;       /* c = alpha dt / h, absolute (not a fraction of c_max)     */
  double alpha;     /* wave speed > 0 (only c enters the discrete operators)    */
  int order_p;      /* upwind order p in 1..5: odd p dissipative (Sec. 6.3),    */
                    /* even p dispersive (Sec. 6.4: eps-dependent SL nodes,     */
                    /* first-order left-biased D^{(p+1)}_1; q = p)              */
  int rk_kind;      /* MGRIT_ERK or MGRIT_SDIRK                                 */
  int rk_order_q;   /* q; 0 means q = p.  ERK q = p only; SDIRK q in 1..5       */
  int m;            /* coarsening factor >= 2                                   */
  int levels;       /* levels incl. the fine one, 2 <= levels <= 16; 0 means    */
                    /* "coarsen until fewer than two time points" (Sec. 6.3)    */
  int nu;           /* CF sweeps in the pre-relaxation F(CF)^nu, 0 <= nu <= 4   */
  double tol;       /* stop when ||r_it|| <= tol ||r_0|| (default 1e-10)        */
  int max_iter;     /* iteration cap (default 30, Sec. 6.3)                     */
  int precision;    /* MGRIT_FP64, MGRIT_MIXED or MGRIT_MIXED_FAST              */
  uint64_t seed;    /* seed of the random initial iterate (SplitMix64)          */
  int inner_cycles; /* MIXED: FP32 V-cycles per FP64 residual; 0: adaptive --  */
                    /* repeat while the FP32 error-equation residual is above   */
                    /* t x the FP64 residual r it corrects, t = max(1e-2, 0.01  */
                    /* tol r_0 / r) (at most 0.1), and still falls by 0.8 per   */
                    /* cycle, at most 16 (checked on the device); the 1e-2      */
                    /* base can be set with the environment MGRIT_INNER_TOL     */
  int coarse_op;    /* coarse-grid operator: MGRIT_COARSE_SL_CORRECTED (0, the  */
                    /* paper's Eq. MOL-SL-corrected-multilevel), MGRIT_COARSE_SL */
                    /* (direct S_p, Sec. 3), MGRIT_COARSE_REDISC (SDIRK only:   */
                    /* the fine method with step m^l dt, Sec. 5)                */
  int coarse_solve; /* correction solve (I - phi D) x = S v of the corrected    */
                    /* operator on every coarse level: MGRIT_SOLVE_DIRECT (0)   */
                    /* or MGRIT_SOLVE_GMRES: GMRES from a zero guess, stopped   */
                    /* once ||b - A x_k|| <= gmres_rtol ||b|| or at gmres_maxit */
                    /* (Sec. 6.1, Sec. 6.3); SL_CORRECTED only, n_x <= 32768    */
  int gmres_maxit;  /* 1..32; 0: 10 for p = 1, 20 otherwise (Sec. 6.3)         */
  double gmres_rtol;/* in (0, 1); 0: 1e-2 (Sec. 6.3)                           */
  int m_coarse;     /* coarsening factor below level 1 (level l >= 1 takes      */
                    /* m_coarse steps per step of level l+1); 0: m.  The        */
                    /* paper's parallel runs use m = 16, m_coarse = 4           */
                    /* (Sec. 6.3.2); level l steps m m_coarse^(l-1) dt          */
} mgrit_params;

/* ---- statistics -------------------------------------------------------- */
typedef struct mgrit_stats {
  int iterations;      /* coarse corrections applied before the stop test    */
  int converged;       /* 1 if ||r|| <= tol ||r_0||                          */
  int levels;          /* levels actually used                               */
  int history_len;     /* entries in rnorm_history                           */
  double rnorm0;       /* ||r_0||                                            */
  double rnorm;        /* last residual norm                                 */
  double conv_factor;  /* rnorm_it / rnorm_{it-1} at the last iteration      */
  double rnorm_history[MGRIT_MAX_HISTORY];
  double ms_total;     /* wall time of mgrit_solve (host clock)              */
  int inner_cycles;    /* MIXED: FP32 V-cycles run in total                  */
  int outer_iterations;/* MIXED: FP64 residual evaluations after the first   */
} mgrit_stats;

typedef struct mgrit_handle mgrit_handle;

/*
 * mgrit_setup -- validate *params, build the level hierarchy and allocate all
 * device buffers on the current CUDA device.
 *   params : host pointer, read only.  Section and equation of each field are
 *            given above.  Derived per-level data (SL shift k_l and eps_l,
 *            phi_l, Phi^m stencil, factorised correction solves) are computed
 *            on the host in FP64 (Sec. 3, Lemma 6.1, Sec. 6.2).
 *   stream : cudaStream_t (as void*) on which all work of the handle runs.
 *   out    : receives the new handle (NULL on failure).
 * Errors: INVALID_ARG (sizes, p outside 1..5, nt % m^(levels-1), stencil wider than
 * nx), UNSTABLE (singular correction matrix), OOM, CUDA.
 */
int mgrit_setup(const mgrit_params* params, void* stream, mgrit_handle** out);

/* Release every buffer of the handle (NULL is accepted). */
int mgrit_destroy(mgrit_handle* h);

/* Static text of an error code. */
const char* mgrit_strerror(int code);

/* Text of the last failing CUDA call of this host thread ("" if none); valid
 * until the next failure on the same thread. */
const char* mgrit_last_error(void);

/*
 * mgrit_set_initial -- set the initial condition u0 (nx values, host or
 * device) and the initial C-point iterate of level 0.  init (host or device,
 * (nt/m + 1) * nx values for time rows n = k m) may be NULL: then the rows
 * k >= 1 are uniform random in [0, 1) from SplitMix64 with params.seed and
 * counter n * nx + i + 1 (Sec. 5.3 setup: random except at t = 0).  Row 0 is
 * always u0.
 */
int mgrit_set_initial(mgrit_handle* h, const double* u0, const double* init);

/*
 * mgrit_relax -- nu CF sweeps on `level` (Sec. 2.2).  F-points are not
 * stored: the F-relaxation is implied by every kernel that reads C-points, so
 * F(CF)^nu amounts to nu C-relaxations, each preceded by the F-relaxation of
 * its interval.  Level 0 acts on the C-point iterate; level l >= 1 on the
 * level's C-point unknowns with the RHS last written by mgrit_residual of
 * level l-1 (zero initial guess if `reset` semantics are wanted: call
 * mgrit_level_io to clear it).  Asynchronous on the handle's stream.
 */
int mgrit_relax(mgrit_handle* h, int level, int nu);

/*
 * mgrit_residual -- F-relax `level` and form the C-point residual
 * r_k = g_{km} + Phi_l u_{km-1} - u_{km}, k = 1..N_l/m (Sec. 2.2; r_0 = 0),
 * store it as the RHS of level+1 (injection) and return ||r||_2 (over all
 * C-points and grid points) in *norm_out (host pointer; may be NULL).
 * Synchronises the stream when norm_out is not NULL.
 */
int mgrit_residual(mgrit_handle* h, int level, double* norm_out);

/*
 * mgrit_coarse_apply -- y = Phi_l x for nvec vectors (device pointers, nvec *
 * nx FP64 each).  level 0: the fine step R_q(-c L_p) (Eq. MOL_M_def);
 * level l >= 1: (I - phi_l D)^{-1} S_p^{(m^l dt)} (Eq. MOL-SL-corrected /
 * multilevel form).  x and y must not overlap.  Asynchronous.
 */
int mgrit_coarse_apply(mgrit_handle* h, int level, const double* d_in, double* d_out, int64_t nvec);

/*
 * mgrit_solve -- full MGRIT solve (two-level if levels == 2, else V-cycles):
 * set_initial(u0, NULL) unless `keep_initial` was requested with
 * mgrit_set_initial beforehand (u0 == NULL keeps the current state), then
 * iterate until ||r_it|| <= tol ||r_0|| or max_iter.  u_out (host or device,
 * may be NULL) receives the (nt/m + 1) * nx level-0 C-point values whose
 * residual was measured last; stats (host, may be NULL) is filled.
 * Returns OK, NOT_CONVERGED or DIVERGED (u_out and stats are still written).
 */
int mgrit_solve(mgrit_handle* h, const double* u0, double* u_out, mgrit_stats* stats);

/*
 * mgrit_solve_async -- the same solve as mgrit_solve, run as one CUDA graph
 * launch without host round trips: the first pre-relaxation and residual,
 * then a device-side loop (a conditional while node) whose body is one
 * MGRIT iteration followed by the stop test (||r|| <= tol ||r_0||,
 * max_iter, divergence) evaluated on the GPU.  The graph is built at the
 * first call and reused.  u0 (host or device, nx; NULL keeps the current
 * initial state) is copied and the random initial iterate generated on the
 * handle's stream.  Returns immediately; at most one solve per handle is in
 * flight.  Not thread safe.
 * mgrit_solve_query -- MGRIT_OK when the solve finished, 1 while running.
 * mgrit_solve_wait  -- wait, then copy the C-points to u_out (host or device,
 * may be NULL) and fill stats (may be NULL); returns the solve's status (OK,
 * NOT_CONVERGED, DIVERGED) like mgrit_solve.
 */
int mgrit_solve_async(mgrit_handle* h, const double* u0);
int mgrit_solve_query(mgrit_handle* h);
int mgrit_solve_wait(mgrit_handle* h, double* u_out, mgrit_stats* stats);

/*
 * mgrit_solve_wait_for -- mgrit_solve_wait bounded on the host: returns
 * MGRIT_ERR_TIMEOUT if the solve has not finished after timeout_s seconds
 * (it stays in flight; wait for it again later), else as mgrit_solve_wait.
 * The paper has no counterpart.
 */
int mgrit_solve_wait_for(mgrit_handle* h, double timeout_s, double* u_out, mgrit_stats* stats);

/*
 * mgrit_vcycle -- one MGRIT iteration without the stop test: coarse
 * correction from the current level-1 RHS (written by mgrit_residual(0)),
 * then the level-0 pre-relaxation F(CF)^nu and residual; *norm_out (host,
 * may be NULL) receives the new ||r||.  Used to compare iterates step by step.
 */
int mgrit_vcycle(mgrit_handle* h, double* norm_out);

/*
 * mgrit_level_rows -- rows row0 .. row0+nrows-1 of a level buffer (field 0:
 * the C-point unknowns, field 1: the RHS, as in mgrit_level_io) against the
 * caller's ptr (nrows * nx doubles): op 0 copies them to ptr (host or
 * device), op 1 copies ptr into them (host or device), op 2 adds ptr
 * (device) to them.  Asynchronous on the handle's stream for device
 * pointers; a host pointer synchronises it.  Unlike mgrit_level_io, op 1 on
 * row 0 of level 0 changes the current buffer only.  Used by time-sharded
 * solves (blocks of CF-intervals on several GPUs, Sec. 6.3.2) to exchange
 * boundary rows and corrections.  Errors: INVALID_ARG (rows outside the
 * buffer, op 2 with a host pointer), CUDA.
 */
int mgrit_level_rows(mgrit_handle* h, int level, int field, int64_t row0, int64_t nrows, double* ptr, int op);

/*
 * mgrit_coarse_correct -- the coarse-grid correction of one MGRIT iteration
 * (Sec. 2.2): solve the level-1 error equation e_{k+1} = Psi e_k + r_{k+1}
 * with the current level-1 RHS (zero initial guess, one cycle over levels
 * >= 1, the coarsest solved sequentially) and add e to the level-0 C-point
 * unknowns (rows 1..nt/m).  Asynchronous.  FP64 handles only (MIXED:
 * MGRIT_ERR_UNSUPPORTED); INVALID_ARG for a one-level handle.
 */
int mgrit_coarse_correct(mgrit_handle* h);

/*
 * mgrit_level_io -- copy a level buffer to or from the caller.
 *   field 0: C-point unknowns of the level (level 0: (nt/m+1) rows; level l:
 *            N_{l+1}+1 rows, N_l = nt/m^l), field 1: RHS g of the level
 *            (N_l + 1 rows, l >= 1).
 *   ptr    : host or device, rows * nx doubles; to_device != 0 copies ptr ->
 *            handle, else handle -> ptr.  *rows_out (may be NULL) gets rows.
 * Synchronises the stream.
 */
int mgrit_level_io(mgrit_handle* h, int level, int field, double* ptr, int to_device, int64_t* rows_out);

/*
 * mgrit_fine_propagate -- GPU sequential time-stepping u_{n+1} = Phi u_n
 * (Eq. one-step-general) for nsteps steps from u0 (host or device, nx) into
 * u_out (host or device, nx), with the fine operator of the handle, in one
 * persistent launch (the vector stays on chip).  This is the baseline MGRIT
 * is measured against.  If `every` > 0 and traj (device) is not NULL, rows
 * n = every, 2 every, ... are also written to traj[(n/every - 1) * nx].
 */
int mgrit_fine_propagate(mgrit_handle* h, const double* u0, double* u_out, int64_t nsteps,
                         int64_t every, double* traj);

/*
 * mgrit_fine_propagate_async -- mgrit_fine_propagate without the final
 * synchronisation: enqueues the sequential stepping on the handle's stream
 * and returns.  d_u0, d_out: device pointers (nx doubles), read / written in
 * stream order; MGRIT_ERR_INVALID_ARG for host pointers.  The caller
 * synchronises the stream.  The paper has no counterpart (it is the
 * baseline's launch form for batches).
 */
int mgrit_fine_propagate_async(mgrit_handle* h, const double* d_u0, double* d_out, int64_t nsteps);

/*
 * mgrit_output_all -- every time point of the current level-0 iterate:
 * row n of d_all (device, (nt + 1) x nx doubles, row-major) is u_n, the
 * C-points u_{km} as they stand and the F-points u_{km+j} regenerated by
 * F-relaxation from them (Sec. 2.2), all intervals at once.  Call it after
 * a solve (or mgrit_set_initial).  MGRIT_ERR_INVALID_ARG for a host pointer
 * or before any iterate exists.
 */
int mgrit_output_all(mgrit_handle* h, double* d_all);

/*
 * mgrit_level_info -- host-side derived data of a level (no GPU work):
 * out[0] = steps N_l, out[1] = SL shift k_l, out[2] = eps_l, out[3] = phi_l
 * (phi_p for q != p), out[4] = phi_q (0 when q = p), out[5] = composite
 * stencil taps (level 0, ERK) or the level's time step in units of dt
 * (coarse levels: m m_coarse^(l-1)), out[6] = chunk length of the in-block solves
 * (level 0, ERK: outputs per thread of the composite-stencil kernel, and
 * out[4] = 1 when its persistent form runs; level 0, SDIRK: out[4] = 2 when
 * the segmented FP64 kernel runs the level's relaxations -- one CTA per
 * interval, 128 points per thread -- and out[5] = 1 when MIXED inner
 * cycles run the FP32 segmented kernel; MGRIT_SDIRK_SEG=0 / 1 disables /
 * forces both where they apply),
 * out[7] = CTAs per vector (thread-block cluster size) of the level's step
 * kernel (coarse levels; level 0 for SDIRK).  The step kernels' geometry is
 * measured at setup among the candidates that fit (cached per shape in the
 * process, and in the file MGRIT_AUTOTUNE_CACHE names); MGRIT_AUTOTUNE=0
 * takes the best-scored candidate unmeasured, MGRIT_GEOM="C:P" forces C CTAs
 * per vector and chunk length P where that geometry fits, MGRIT_STENCIL=R
 * (or R + 16: the persistent form) the level-0 stencil tile.
 */
int mgrit_level_info(const mgrit_handle* h, int level, double out[8]);

/*
 * mgrit_gmres_stats -- GMRES work on coarse level `level` (>= 1) since setup:
 * out[0] = iterations summed over all correction solves, out[1] = solves
 * (zeros when the level solves directly).  Waits for the handle's stream.
 * Errors: INVALID_ARG (level out of range, out NULL), CUDA.
 */
int mgrit_gmres_stats(mgrit_handle* h, int level, int64_t out[2]);

/* Number of CUDA kernels this handle launched since setup (kernel-launch
 * counter maintained by the library). */
int64_t mgrit_launch_count(const mgrit_handle* h);

/*
 * mgrit_profile -- enable (1) or disable (0) per-kernel timing with CUDA
 * events recorded on the handle's stream around every launch; enabling
 * clears the counters.  Not in the paper: measurement support.
 * mgrit_profile_read -- out[3c+0] launches, out[3c+1] summed device ms,
 * out[3c+2] algorithmic flops (2 per multiply-add the kernel must do) for
 * category c = 0 level-0 composite stencil, 1 coarse step kernel (all
 * levels), 2 reductions, 3 sequential stepping, 4 + l coarse step kernel on
 * level l (l = 1..14, the last of these slots collects deeper levels),
 * 19 the FP32 level-0 kernels of MIXED inner cycles; 20 categories, out has
 * 60 entries.  Synchronises the stream.
 */
int mgrit_profile(mgrit_handle* h, int enable);
int mgrit_profile_read(mgrit_handle* h, double out[60]);

/*
 * mgrit_residual_noalloc -- the level-0 C-point residual of mgrit_residual
 * (level 0) and its l2 norm, for callers that cannot allocate device memory
 * when they need it: code recording a CUDA graph by stream capture (device
 * allocation is not a capturable operation) and applications whose device
 * memory belongs to a pool or caching allocator that must not be bypassed.
 * The paper has no counterpart; this is an interface convenience.
 *
 * It takes no handle (mgrit_setup allocates) and allocates nothing, on the
 * device or the host heap.  Its scratch (the per-CTA partial sums of the
 * norm) lives in one static device array of 65536 + 32 doubles (512 KB) that
 * every GPU loading the library holds until the process exits.
 *   params  : host; fields nx, cfl, order_p, rk_order_q (0 or p), m are used;
 *             rk_kind must be MGRIT_ERK, precision MGRIT_FP64 and order_p
 *             odd (1, 3 or 5); other orders return MGRIT_ERR_INVALID_ARG.
 *             The composite stencil Phi^m is folded modulo nx; if it still
 *             has more than 1024 taps the call returns MGRIT_ERR_UNSUPPORTED.
 *   d_uC    : device, rows * nx C-point values u_{k m}, k = 0..rows-1.
 *   rows    : >= 2; (rows - 1) * ceil(nx / 1024) must not exceed 65536
 *             (nx >= 1024; ceil(nx / 512) or ceil(nx / 256) below), else
 *             MGRIT_ERR_INVALID_ARG and nothing runs.
 *   d_r     : device, (rows - 1) * nx outputs r_k = Phi^m u_{(k-1)m} - u_{km}
 *             (the fine map applied m times to the previous C-point, minus
 *             the C-point), k = 1..rows-1; must not overlap d_uC.
 *   norm_out: host, receives ||r||_2; NULL skips the copy (the call is then
 *             fully asynchronous).  With norm_out the stream is synchronised,
 *             which a stream capture does not allow: while the stream is
 *             being captured pass NULL (d_r is still written; the norm is
 *             then not returned).
 *   stream  : cudaStream_t as void*.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current) and may load the
 * library's device code; make that first call before any stream capture.
 * Every call shares the one array and overwrites its contents, so calls
 * whose kernels overlap on the GPU (different streams, or different host
 * threads) race on it: serialise them.
 */
int mgrit_residual_noalloc(const mgrit_params* params, const double* d_uC, int64_t rows, double* d_r,
                           double* norm_out, void* stream);

/* ---- batched and served solves ----------------------------------------- */
/*
 * Many independent advection problems of different sizes (the batched
 * workload) run as graph-resident solves captured into one CUDA graph and
 * launched together, so their kernels share the GPU and no solve waits on
 * the host between iterations.
 * The paper solves one problem at a time; batching is an interface layer.
 */
typedef struct mgrit_batch mgrit_batch;

/* Device bytes mgrit_setup allocates for *p (admission estimate), or -1. */
int64_t mgrit_estimate_bytes(const mgrit_params* p);

/* count solves with per-solve parameters params[0..count) (host); the
 * hierarchies are set up on nstreams internal streams (and the sequential
 * baseline runs over them).  Allocates every hierarchy up front. */
int mgrit_batch_create(const mgrit_params* params, int64_t count, int nstreams, mgrit_batch** out);
/* Solve all: u0s[i] (host or device, params[i].nx values).  stats (host, count
 * entries, may be NULL).  Every solve of the batch is one independent branch
 * of a single CUDA graph (captured at the first call), so the whole batch is
 * one graph launch.  Returns OK, or the first NOT_CONVERGED / DIVERGED
 * status among the solves (all solves still ran). */
int mgrit_batch_solve(mgrit_batch* b, const double* const* u0s, mgrit_stats* stats);
/* C-points of solve i ((nt/m + 1) * nx values, host or device). */
int mgrit_batch_get(mgrit_batch* b, int64_t i, double* u_out);
/* Sum of nx * nt over the batch. */
int64_t mgrit_batch_dof(const mgrit_batch* b);

/*
 * mgrit_batch_sequential -- the GPU sequential-stepping baseline of a batch:
 * solve i stepped nt_i times from d_u0s[i] into d_outs[i] (device, nx_i
 * doubles each), all solves enqueued over the batch's stream pool at once,
 * then synchronised.  The paper has no counterpart.
 */
int mgrit_batch_sequential(mgrit_batch* b, const double* const* d_u0s, double* const* d_outs);
int mgrit_batch_destroy(mgrit_batch* b);

typedef struct mgrit_request_result {
  double start_s;     /* admission time (s from the start of mgrit_serve)   */
  double finish_s;    /* completion time                                   */
  double latency_ms;  /* finish - arrival                                  */
  int iterations;
  int status;         /* MGRIT status; 1 = never admitted (time limit)     */
} mgrit_request_result;

typedef struct mgrit_serve_stats {
  int64_t arrived, admitted, completed, failed, rejected;
  int64_t backlog_end;   /* requests not admitted when the run ended         */
  int64_t max_backlog;   /* largest queue of arrived, not admitted requests  */
  int64_t max_mem_bytes; /* peak admitted device memory (estimate)           */
  int max_inflight, pad;
  double dof_completed;  /* sum of nx * nt over completed requests           */
  double wall_s;
  double setup_s;        /* host time spent setting up admitted requests    */
} mgrit_serve_stats;

/*
 * mgrit_serve -- replay a stream of solve requests with continuous batching:
 * request i (params[i], initial condition u0s[i] on the host) arrives at
 * arrival_s[i] seconds (non-decreasing) after the call starts; arrived
 * requests are admitted while fewer than max_inflight solves run and the
 * estimated device memory of the running solves stays within
 * hbm_budget_bytes -- the first that fits among the 64 oldest waiting
 * requests, except that a request waiting longer than 2 s is not overtaken
 * -- and each admitted request gets its own hierarchy (set up on admission,
 * freed on completion) and runs as a graph-resident solve overlapping the
 * others on the GPU.  No launch geometry is timed while serving: setups
 * use geometries measured earlier in the process (mgrit_setup of the same
 * shapes before the call, on an idle GPU) or the best-scored candidate.  Returns when all
 * requests finished or after time_limit_s (running solves are drained,
 * unadmitted ones keep status 1).  u_outs (may be NULL, as may each
 * u_outs[i]) receives request i's C-points ((nt/m + 1) * nx values, host or
 * device).  results (host, count entries) and st (host, may be NULL) are
 * filled.
 */
int mgrit_serve(const mgrit_params* params, const double* const* u0s, double* const* u_outs,
                const double* arrival_s, int64_t count, int64_t hbm_budget_bytes, int max_inflight,
                double time_limit_s, mgrit_request_result* results, mgrit_serve_stats* st);

#ifdef __cplusplus
}
#endif
#endif /* MGRIT_H_ */
