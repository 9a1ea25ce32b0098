/*
 * hz.h -- C ABI of the GB300 interpolated pseudodifferential Helmholtz solver.
 *
 * The library solves the periodic finite-difference Helmholtz system
 *     P_N u = f,   P_N u = gamma^2 Lap_h u + (omega^2 + i omega a) u
 * (Eqn. 001 discretised as in Section 5 "Numerical experiments": second-order
 * centred differences, periodic boundaries) with restarted GMRES, right- and
 * flexibly preconditioned by the interpolated pseudodifferential operator
 *     Q_M v = sum_k w_k(x) IFFT( q_k(xi) FFT(v) ),
 *     q_k(xi) = 1 / (omega^2 + i omega a_k - gamma_k^2 |xi|^2)
 * (Eqn. 021, Eqn. 103, and Eqn. 403/405 with the complex wave speed
 * gamma = c (1 - i zeta) of Eqn. Complex_wave_speed, Section 4.4).
 *
 * Conventions shared by every entry point
 *   - Grid: dim 2 or 3, n[0] = Nx (fastest), n[1] = Ny, n[2] = Nz; unit box of
 *     side L with spacing h = L / N per axis; every axis periodic.  Supported
 *     axis lengths: 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 512, 1024,
 *     2048, and with a factor 5 (the grids of the paper's Section 5): 20,
 *     40, 60, 120, 180, 240, 360, 480, 720, 960, 1440, 1920, 2400, 2880,
 *     3600, 4800; z at most 1024.
 *   - Complex vectors are interleaved (re, im).  "c128" = two doubles, "c64" =
 *     two floats.  Several right-hand sides are stored one after another with
 *     stride n = Nx Ny Nz elements.
 *   - Device pointers, unless an entry point says it also takes host memory.
 *     The caller owns every buffer it passes; the library owns what it
 *     allocates (media, plans, their workspace).
 *   - stream: a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Work is enqueued asynchronously unless stated otherwise.
 *   - Every call returns an hz_status; on failure hz_last_error() gives a
 *     thread-local message.  No entry point traps on the device: device-side
 *     failures are reported through a status word that the host reads.
 */
#ifndef HZ_H
#define HZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HZ_OK = 0,
  HZ_ERR_INVALID_ARG = 1,   /* bad pointer, size, option or unsupported grid  */
  HZ_ERR_OOM = 2,           /* device allocation failed                       */
  HZ_ERR_CUDA = 3,          /* a CUDA runtime call failed                     */
  HZ_ERR_NOT_CONVERGED = 4, /* maxit reached; the best iterate is still written */
  HZ_ERR_BREAKDOWN = 5,     /* NaN/Inf in the Krylov recurrence               */
  HZ_ERR_TIMEOUT = 6,       /* a bounded device wait ran out                  */
  HZ_ERR_BUSY = 7,          /* server queue full / HBM budget exhausted       */
  HZ_ERR_MEDIUM = 8         /* c <= 0, zeta < 0, or c != c_o inside the layer  */
} hz_status;

typedef struct {
  int dim;      /* 2 or 3                                  */
  int n[3];     /* Nx, Ny, Nz (Nz ignored when dim == 2)   */
  double L;     /* side of the periodic box, > 0           */
} hz_grid;

/* Interpolation set-up (Section 4.1, Lemma 3, Section 4.4).
 *   M          number of real wave-speed nodes, equispaced on [c_min, c_max];
 *              c_o is forced to be a node when a layer exists (two equispaced
 *              segments when c_o lies strictly inside the range).  M = 1 gives
 *              the single-node Q_1 of Eqn. OneInterpPoint at c_o.
 *   Mt         number of layer nodes c_o (1 - i zeta_m), zeta_m = m zeta_max / Mt.
 *   c_o        background speed; c must equal c_o wherever zeta > 0.
 *   zeta_max   <= 0: take max(zeta) of the medium.
 *   alpha      node symbols use the damping a_k = a_node + alpha * omega.
 *   a_node     see alpha (the paper's a(c) assumption, Section 4, with one
 *              value for every node).
 *   symbol_kind 0: |xi|^2 = sum (2 pi k / L)^2 (Eqn. 021);
 *               1: the finite-difference symbol sum (4/h^2) sin^2(pi k / N).
 *   Ma         0 or 1: the damping of every node symbol is a_node + alpha w
 *              (a follows c, Eqn. Intro02).  >= 2: bivariate interpolation in
 *              (c, a), the extension Section 6 names for damping that does
 *              not follow the wave speed: Ma damping nodes a_j equispaced on
 *              [min a, max a] (one node when a is constant or NULL), node
 *              k = s Ma + j with speed node s and damping a_j + alpha w, and
 *              weights = speed weight x hat in a (up to 4 per point).
 *              K = (M + Mt) Ma must stay <= 64.
 *   basis      0: piecewise-linear hats in c (Eqn. 405); 1: piecewise
 *              quadratic Lagrange polynomials on elements of two intervals
 *              (the higher-order basis of Section 6; M odd, and with c_o
 *              inside the range each of its two segments gets an even
 *              number of intervals); 2: piecewise cubic Hermite in c (the
 *              other basis Section 6 names): on [c_m, c_m+1] the planes of
 *              q(c_m) and q(c_m+1) take h00(t), h01(t) and M extra planes
 *              with the symbol's derivative dq/dc = 2 c |xi|^2 q^2 at the
 *              real nodes take h h10(t), h h11(t) (K = M + Mt + M).  Layer
 *              points keep the hats in zeta.  basis 1 and 2 are univariate
 *              only (Ma <= 1).
 * Fields added later (Ma, basis) read as 0 when a caller zero-fills the
 * struct, which keeps the univariate piecewise-linear method.           */
typedef struct {
  int M;
  int Mt;
  double c_o;
  double zeta_max;
  double alpha;
  double a_node;
  int symbol_kind;
  int Ma;
  int basis;
} hz_interp;

/* Solver options.
 *   precision  0: plain FP64 path (complex128 preconditioner, GMRES storing
 *                 no Z: u = u0 + Q(V y));
 *              1: complex64 preconditioner inside flexible GMRES; Arnoldi,
 *                 operator and residuals stay FP64.
 *   restart    m, the Krylov dimension per cycle (1..128).
 *   tol        stop when ||f - P_N u||_2 / ||f||_2 <= tol (true residual).
 *   maxit      cap on the total number of Arnoldi steps.
 *   graphs     1: capture each full Arnoldi cycle once as a CUDA graph and
 *              replay it (worth it for small grids, where launches cost as
 *              much as the kernels); 0: launch step by step.
 *   no_precond 1: plain GMRES(m) on P_N u = f without the preconditioner,
 *              all in FP64 (the unpreconditioned baseline the paper compares
 *              against in Section 5); 0: preconditioned by Q_M.
 *   left       1: the paper's left preconditioning (Eqn. MainDiscretePrecond):
 *              GMRES(m) on Q_M P_N u = Q_M f, each Arnoldi vector
 *              Q_M (P_N v) (the stencil in FP64, Q_M in the precision
 *              above), u += V y, and the stopping test (and the history) on
 *              the preconditioned residual ||Q_M (f - P_N u)|| / ||Q_M f||,
 *              as the paper's GMRES runs report it; hz_solve_stats still
 *              reports the true residual.  0: right / flexible (default).
 *              Ignored with no_precond.                                 */
typedef struct {
  int precision;
  int restart;
  double tol;
  int maxit;
  int graphs;
  int no_precond;
  int left;
} hz_solver_opts;

typedef struct {
  int iters;               /* Arnoldi steps taken                          */
  int restarts;            /* cycles run                                   */
  int status;              /* hz_status of this right-hand side            */
  int converged;           /* 1 when the true residual met tol             */
  double rel_true_resid;   /* ||f - P_N u|| / ||f|| in FP64 at return      */
  double rel_est_resid;    /* last Givens estimate                          */
  float ms_total;          /* wall time of the solve on the stream (events) */
  /* Phase times of this solve call (all of its right-hand sides together),
   * filled only while hz_profile_enable(1) is on and for launches made step
   * by step (a captured cycle graph carries no events: with opts.graphs = 1
   * they cover the launches outside the graph); 0 otherwise.            */
  float ms_precond;        /* preconditioner passes: FFTs, symbol, weighted sum */
  float ms_stencil;        /* operator P_N: Arnoldi products and residuals  */
  float ms_arnoldi;        /* CGS2 dots and updates, Givens, norms, u update */
  double model_bytes_precond; /* algorithmic bytes of those preconditioner
                               passes (each input read once, each output
                               written once; planes only on the rows / slabs
                               that use them)                              */
} hz_solve_stats;

typedef struct hz_medium hz_medium;
typedef struct hz_plan hz_plan;

/* Thread-local description of the last failure in this thread. */
const char* hz_last_error(void);

/* Library version string. */
const char* hz_version(void);

/* Device allocator used for media and plans.  alloc(bytes, ctx) returns a
 * device pointer or NULL; release(ptr, ctx) frees it.  Passing NULL for both
 * restores cudaMalloc / cudaFree.  Not thread-safe against concurrent
 * create/plan calls. */
hz_status hz_set_allocator(void* (*alloc)(size_t bytes, void* ctx),
                           void (*release)(void* ptr, void* ctx), void* ctx);

/* Build a medium (Section 4.4 node table, per-point interpolation records and
 * gamma^2 of Eqn. Complex_wave_speed) from HOST arrays of n doubles each,
 * indexed [z][y][x].  c: wave speed (> 0); zeta: layer profile (>= 0, NULL =
 * no layer); a: operator damping of Eqn. 001 (NULL = 0).  The arrays are
 * copied; the call returns after the medium is ready.  Axis lengths: 8, 12,
 * 16, 24, 32, 48, 64, 96, 128, 192, 256, 512, 1024, 2048 and the lengths with
 * a factor 5 listed at the top of this file (z <= 1024); fewer
 * than 2^31 points.
 * With interp->Ma >= 2 or interp->basis >= 1 the per-point record is up to
 * four (node, weight) pairs (52 bytes per point) instead of (segment, t).
 * Errors: HZ_ERR_INVALID_ARG (grid, options: Ma < 0, basis not 0/1/2, basis
 * 1 or 2 with Ma >= 2, basis 1 with an even M, more than 64 planes), HZ_ERR_MEDIUM (c <= 0,
 * zeta < 0, NaN, c != c_o in the layer, too few nodes), HZ_ERR_OOM,
 * HZ_ERR_CUDA. */
hz_status hz_create_medium(const hz_grid* grid, const double* c, const double* zeta,
                           const double* a, double omega, const hz_interp* interp,
                           hz_medium** out);

/* Node table of a medium: K = number of symbol planes, M real nodes, Mt layer
 * nodes (K = (M + Mt) Ma, node k = s Ma + j in the bivariate form);
 * gamma_re/gamma_im/a_k receive K values each (may be NULL);
 * c_min/c_max over the grid. */
hz_status hz_medium_info(const hz_medium* med, int* K, int* M, int* Mt, double* gamma_re,
                         double* gamma_im, double* a_k, double* c_min, double* c_max);

hz_status hz_destroy_medium(hz_medium* med);

/* A plan owns the workspace to apply Q_M (Eqn. 103 / 403: the transformed
 * input and K symbol planes per right-hand side) and to run the restarted
 * GMRES of Section 5 ("GMRES implementation": the Krylov basis V of m + 1
 * c128 vectors, for precision 1 the m c64 preconditioned vectors Z of
 * flexible GMRES, and the small Hessenberg systems) for up to max_nrhs
 * right-hand sides at once on one medium.  The medium must outlive the plan
 * and its device must be current.  hz_plan_bytes reports the size.
 * Errors: HZ_ERR_INVALID_ARG (precision or no_precond not 0 / 1, restart
 * outside 1..128, tol <= 0, maxit < 1, max_nrhs < 1), HZ_ERR_OOM. */
hz_status hz_plan_create(hz_medium* med, const hz_solver_opts* opts, int max_nrhs,
                         hz_plan** out);

/* Autotuner (the paper has no counterpart; it tunes this implementation's
 * launch shapes).  Times candidate launch shapes of the kernels that dominate
 * a solve on the plan's own buffers with CUDA events on `stream`: blocks per
 * SM and vectors per block of the CGS2 dot kernel, blocks per SM of the CGS2
 * update, nodes per block and columns per thread of the last-axis symbol
 * pass, and whether the x-inverse pass accumulates the weighted sum as it
 * goes, transforms the planes in place and gathers the sum afterwards, or
 * transforms each (row, node) line on its own and adds it into the output.  The choice is stored
 * in the plan and cached per (grid, K, max_nrhs, restart, precision) for the
 * process; later plans with the same key reuse it without timing.
 * Synchronous; overwrites the plan's work arrays (call before solving). */
typedef struct {
  int dots_bps, dots_vc, upd_bps, syminv_kpb;
  int cached;               /* 1: taken from the process cache, no timing  */
  float dots_us, dots_us_default;     /* chosen vs default shape           */
  float upd_us, upd_us_default;
  float apply_us, apply_us_default;   /* whole preconditioner apply        */
  int rowinv_mode;          /* x-inverse pass: 0 by grid size, 1 in place
                               then a gather of the weighted sum, 2 fused,
                               3 one line per (row, node) in use, added
                               into the cleared output (bitwise
                               reproducible with the two-node records; with
                               the up to four weights of Ma >= 2 or
                               basis 1 the order of the additions can
                               change the last bits, and the autotuner
                               leaves this form out for such media)        */
  int col_pair;             /* complex64 symbol pass: 1 two columns per
                               thread in packed FP32, 2 the same in blocks
                               of half the size, 0 one column              */
} hz_tune_report;

hz_status hz_plan_autotune(hz_plan* plan, void* stream, hz_tune_report* report);

/* Sets the plan's launch shapes from a report (e.g. one saved from an
 * earlier hz_plan_autotune): dots_vc in {2, 4, 8}, dots_bps in 1..4, upd_bps
 * in 1..8, syminv_kpb in {1, 2, 4}, rowinv_mode in {0, 1, 2, 3}, col_pair in
 * {0, 1, 2}; the timing
 * fields are ignored.  HZ_ERR_INVALID_ARG for any other value. */
hz_status hz_plan_set_tune(hz_plan* plan, const hz_tune_report* report);

/* Bytes of device memory the plan holds. */
hz_status hz_plan_bytes(const hz_plan* plan, size_t* bytes);

hz_status hz_destroy_plan(hz_plan* plan);

/* y = P_N x (Eqn. 001 discretised as in Section 5: the 5-point (2D) or
 * 7-point (3D) centred second difference, periodic, with gamma^2 of
 * Eqn. Complex_wave_speed in the layer) for nrhs vectors, x != y, device
 * pointers.  The arithmetic is FP64 in both precisions, as the Krylov method
 * needs it: precision 0 reads x as c128; precision 1 reads x as c64 (the
 * form in which flexible GMRES stores its preconditioned vectors, widened
 * exactly to FP64).  y is always c128.  Errors: HZ_ERR_INVALID_ARG for null
 * or aliasing pointers, nrhs outside 1..max_nrhs, precision not 0 / 1, or a
 * current device other than the medium's. */
hz_status hz_apply_operator(hz_plan* plan, const void* x, void* y, int nrhs, int precision,
                            void* stream);

/* y = Q_M x for nrhs c128 device vectors (x may equal y).  precision 0
 * computes in complex128, 1 in complex64 (input rounded to c64, output
 * widened to c128).  Eqn. 103 / 403 with one forward FFT, K symbol
 * multiplies each followed by an inverse FFT, and the weighted sum. */
hz_status hz_apply_preconditioner(hz_plan* plan, const void* x, void* y, int nrhs,
                                  int precision, void* stream);

/* Allocation-free variant of hz_apply_preconditioner (the paper has no
 * counterpart; this is a deployment aid).  y = Q_M x for nrhs c128 device
 * vectors on a medium, without a plan: the transformed input and the K
 * symbol planes live in one fixed device array of 32 MiB that the library
 * image carries (every GPU that loads the library holds it until exit).
 * For callers that cannot allocate device memory when they need the apply:
 * code inside another runtime that owns the GPU's memory through its own
 * pool, or a latency-bound loop that cannot afford cudaMalloc / cudaFree,
 * which synchronise the device.  This call allocates nothing.
 *   - Needs nrhs * n * (K + 1) * (16 for precision 0, 8 for precision 1)
 *     bytes (plus 256 for alignment) <= 32 MiB, e.g. one 256 x 256 right-hand
 *     side with K = 16 in complex128, or one 512 x 512 with K <= 15 in
 *     complex64; larger requests return HZ_ERR_INVALID_ARG with the sizes.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, and caches it for
 *     that device's current CUDA context; a call made after the context
 *     was destroyed and recreated (cudaDeviceReset, primary context
 *     released and retained again) looks the address up again.  Make the
 *     first call on each device and context before any stream capture.
 *   - The medium's device must be the current device
 *     (HZ_ERR_INVALID_ARG otherwise).
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (different streams, or several host threads) race and corrupt each
 *     other's results; serialise them.  No part of the array has to start
 *     at zero: each call writes every element it later reads.
 *   - Arguments, layout and precision as for hz_apply_preconditioner. */
hz_status hz_apply_preconditioner_noalloc(const hz_medium* med, const void* x, void* y, int nrhs,
                                          int precision, void* stream);

/* Solve P_N u = f (Eqn. 001 discretised as in Section 5) for nrhs
 * right-hand sides with the restarted GMRES of Section 5 ("GMRES
 * implementation"; the paper preconditions from the left, this library from
 * the right, flexibly for precision 1, so that tol applies to the true
 * unpreconditioned residual): CGS2 Arnoldi in FP64, complex Givens
 * rotations, true-residual check after each cycle whose estimate reached
 * tol.  f and u are c128 arrays of
 * nrhs * n elements in device OR host memory (host buffers are staged
 * through the plan); u holds the initial guess on entry.  stats receives
 * nrhs entries (may be NULL).  Synchronous: returns when the solve is done.
 * Returns HZ_OK when every right-hand side converged, HZ_ERR_NOT_CONVERGED
 * (u still holds the last iterate) or HZ_ERR_BREAKDOWN otherwise. */
hz_status hz_gmres_solve(hz_plan* plan, const void* f, void* u, int nrhs,
                         hz_solve_stats* stats, void* stream);

/* hz_gmres_solve that also returns the residual history: history (host,
 * nrhs * history_len doubles) receives, for right-hand side b and Arnoldi
 * step s < history_len (counted across restarts), the Givens estimate of
 * ||f - P_N u_s|| / ||f|| after that step (the quantity plotted against
 * the GMRES iteration in Section 5); entries past the last step are NaN.
 * Runs step by step (opts.graphs is ignored for this call). */
hz_status hz_gmres_solve_history(hz_plan* plan, const void* f, void* u, int nrhs,
                                 hz_solve_stats* stats, double* history, int history_len,
                                 void* stream);

/* The Hessenberg matrix of the last Arnoldi cycle of right-hand side rhs in
 * the plan's most recent solve, before the Givens rotations: column j holds
 * h_{0..j+1, j} of the (F)GMRES relation P_N Z_J = V_{J+1} H, i.e. of the
 * right-preconditioned operator P_N Q_M (or P_N alone with no_precond), so
 * the eigenvalues of its square part are Ritz values of that operator (the
 * spectral estimates compared with Tables 2-6).  H: host array of
 * (restart + 1) * restart complex128 entries, written column by column with
 * leading dimension restart + 1; *cols receives the number of columns J
 * (0 if rhs did not run in the final cycle).  Synchronous. */
hz_status hz_plan_hessenberg(const hz_plan* plan, int rhs, void* H, int* cols);

/* ---- serving ----------------------------------------------------------
 * A server queues solve requests and admits them onto the GPU as slots and
 * device memory free up (admission by each request's device footprint
 * against hbm_budget, first fit in arrival order, with aging so that small
 * requests cannot overtake a large one without bound).  Each admitted request
 * runs medium set-up, plan, (F)GMRES solve and read-back on its own
 * non-blocking stream and host worker, so the work of concurrent requests
 * overlaps on the device; allocations use the stream-ordered pool.  Every
 * reduction is fixed-order and per request: a result is the same alone and
 * in any mix.  The paper solves one problem at a time; this is the
 * continuous-batching layer around its method. */
typedef struct {
  size_t hbm_budget;   /* device bytes admitted requests may hold; 0 = 80% of free memory */
  int max_slots;       /* requests on the GPU at once (1..64)                            */
  int max_queue;       /* queued requests before hz_submit returns HZ_ERR_BUSY             */
  int device;          /* CUDA device the server uses                                      */
  int autotune;        /* launch shapes of a served plan: 0 the autotuner's process cache
                          entry for the request's grid, K, restart and precision (nearest
                          right-hand-side count; no timing), defaults when there is none;
                          1 the same, and hz_plan_autotune on a miss (once per key, on the
                          request's stream); -1 the defaults                               */
  int max_bypass;      /* aging: a queued request that later arrivals have been admitted
                          ahead of this many times is not overtaken again; 0 = 2 max_slots */
  int batch_slots;     /* 0: each request runs alone.  1..64: continuous batching of
                          requests on the same problem (grid, medium arrays, omega, interp
                          and solver options; only f differs): a request with at most
                          batch_slots right-hand sides starts a batched solve of
                          batch_slots slots or joins a running one at its next restart
                          boundary, and leaves at the boundary after its last right-hand
                          side finished; the others keep iterating.  A right-hand side's
                          result does not depend on which requests share the batch.
                          Right / flexible preconditioning only (opts.left = 0).         */
  int order;           /* admission order: 0 the first queued request (arrival order)
                          that fits the budget; 1 the fitting request with the smallest
                          footprint first (about the least work), so that short requests
                          do not queue behind long ones; aging (max_bypass) bounds how
                          often a request can be overtaken in both orders.               */
} hz_server_opts;

typedef struct {
  hz_grid grid;
  const double* c;        /* host, n values (copied by hz_submit)  */
  const double* zeta;     /* host or NULL                          */
  const double* a;        /* host or NULL                          */
  double omega;
  hz_interp interp;
  hz_solver_opts opts;
  int nrhs;
  const void* f;          /* host c128, nrhs * n (copied)          */
} hz_request;

typedef struct {
  long long submitted, completed, failed, rejected;
  int active, queued, max_active;
  size_t hbm_in_use, hbm_budget;
  double p50_ms, p99_ms, mean_ms;  /* submit-to-completion latency of finished requests */
  double rhs_per_s;                /* right-hand sides solved per second since creation  */
  long long batch_joins;           /* requests that joined a running batched solve       */
} hz_server_stats;

typedef struct hz_server hz_server;

/* Device bytes a request holds while it runs (medium + plan), the quantity
 * admission compares against hbm_budget.  K is taken as M + Mt. */
size_t hz_request_footprint(const hz_grid* grid, const hz_interp* interp,
                            const hz_solver_opts* opts, int nrhs, int has_a);

hz_status hz_server_create(const hz_server_opts* opts, hz_server** out);

/* Copies the request and queues it; returns at once with a ticket.
 * HZ_ERR_BUSY when the queue is full or the request alone exceeds the
 * budget; HZ_ERR_INVALID_ARG for a malformed request. */
hz_status hz_submit(hz_server* s, const hz_request* req, uint64_t* ticket);

/* *done = 0 while the request is queued or running.  When done, copies the
 * solution (nrhs * n c128, host; u_out may be NULL) and nrhs stats entries
 * (may be NULL), releases the ticket and returns the request's status. */
hz_status hz_poll(hz_server* s, uint64_t ticket, int* done, void* u_out, hz_solve_stats* stats);

/* Blocks until the request is done (then hz_poll it) or timeout_s passes
 * (HZ_ERR_TIMEOUT). */
hz_status hz_server_wait(hz_server* s, uint64_t ticket, double timeout_s);

hz_status hz_server_get_stats(hz_server* s, hz_server_stats* out);

/* Drops queued requests, waits for the running ones, frees the server. */
hz_status hz_server_destroy(hz_server* s);

/* ---- measurement ------------------------------------------------------
 * Per-phase timing with CUDA events recorded on the stream each kernel is
 * launched on, plus the algorithmic bytes and flops of every launch (the
 * compulsory traffic of the phase: each input read once, each output written
 * once; the symbol planes only for the rows that use them).  Phases:
 * fft_row_fwd, fft_line, fft_fused, fft_row_inv_acc, stencil, cgs2_dots,
 * cgs2_update, givens, solution_update, residual, norm.
 * hz_profile_enable(1) turns recording on for the whole process (it adds two
 * event records per launch); hz_profile_read waits for the recorded events,
 * fills up to max entries and optionally resets the counters.  With the
 * environment variable HZ_NVTX=1 every phase is also an NVTX range of the
 * same name, for timeline tools (read once per process). */
typedef struct {
  char name[24];
  long long launches;
  double ms;      /* summed event time                        */
  double bytes;   /* summed algorithmic bytes                  */
  double flops;   /* summed algorithmic floating-point ops     */
} hz_phase_stats;

hz_status hz_profile_enable(int on);
hz_status hz_profile_read(hz_phase_stats* out, int max, int* count, int reset);

/* Number of kernels this library has launched in this process. */
unsigned long long hz_launch_count(void);

/* Measures this GPU's FP64 FMA throughput (GFLOP/s, 2 flops per FMA) with a
 * kernel of independent FMA chains filling every SM for about 0.1 s; the
 * denominator for the FP64-bound Krylov kernels.  Synchronous. */
hz_status hz_measure_fp64_peak(double* gflops);

#ifdef __cplusplus
}
#endif

#endif /* HZ_H */
