/*
 * fct.h -- C ABI of the GB300 sparse Fast Chebyshev Transform hot path.
 *
 * Method (Jones, Letourneau, Morse, Langston, "A Sparse Fast Chebyshev
 * Transform for High-Dimensional Approximation"):
 *   given a known multi-index support S (N columns) and an L-grid of K tensor
 *   Chebyshev grids (Sec. 3.2, Algorithm 1), sample f on every grid, take each
 *   grid's multi-dimensional DCT (Algorithm 3), and solve
 *     c* = argmin_c || F f - A c ||_2                       (Sec. 3.4)
 *   where A stacks one alias block per grid (Eq. (L-grid_A_mat)) whose
 *   entries come from the Chebyshev aliasing relation (Lemma (lem:aliasing),
 *   Eq. (aliasing_matrix_nd_diff)), by the CG method on the least-squares
 *   problem (CGLS).
 *
 * Grid and DCT kinds (fct_options.grid_kind):
 *   FCT_GRID_EXTREMA (default): Chebyshev extrema points
 *     x_j = cos(pi j/(n-1)), j = 0..n-1, with an interpolating DCT-I per axis,
 *     so that degree m folds to fold_n(m) = r <= n-1 ? r : 2(n-1)-r,
 *     r = m mod 2(n-1), with entry 1.
 *   FCT_GRID_FIRST_KIND: the paper's own form, first-kind points
 *     x_j = cos((j+1/2) pi/n) (Eq. (chebyshev_grid)), the 1/n DCT-II
 *     quadrature of Eq. (quad_1D) and the signed entries 1, +-1/2, 0 of
 *     Eq. (aliasing_matrix_1d).
 * An axis with n == 1 holds one sample at a caller-given node xi; a column's
 * entry on such a grid carries the factor prod_{i: n_i = 1} T_{m_i}(xi_i).
 *
 * Conventions for every function:
 *   - Return value: fct_status (FCT_OK == 0).  No function throws or aborts.
 *     On failure fct_last_error() returns a thread-local message.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device (e.g. a torch tensor's data_ptr).
 *   - A stream argument is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Device work is asynchronous on that stream unless a
 *     function says it synchronises.
 *   - The caller owns every buffer it passes; the library keeps no pointer to
 *     caller memory after a call returns.  A plan owns its device tables and
 *     Krylov workspace.  One plan must not run two executes at once.
 *   - Support order in equals coefficient order out.
 *   - Layouts: support uint16[N][D]; sizes int32[K][D]; nodes double[K][D];
 *     samples double[M], grid l's tensor of shape sizes[l] in row-major order
 *     (last axis fastest), grids concatenated in order, M = sum_l prod_i n_{l,i}.
 */
#ifndef FCT_H
#define FCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FCT_OK = 0,
  FCT_ERR_INVALID_ARG = 1,  /* malformed sizes, support, options or pointers   */
  FCT_ERR_RANK = 2,         /* plan rejected by its rank check (kappa_max)      */
  FCT_ERR_NOCONV = 3,       /* iteration cap reached; best iterate is written   */
  FCT_ERR_TIMEOUT = 4,      /* a bounded device-side wait expired               */
  FCT_ERR_OOM = 5,          /* device allocation failed                          */
  FCT_ERR_NONFINITE = 6,    /* NaN/Inf met in the samples or a reduction         */
  FCT_ERR_CUDA = 7,         /* any other CUDA runtime error                      */
  FCT_ERR_NO_DEVICE = 8     /* no usable CUDA device                             */
} fct_status;

enum { FCT_FP64 = 0, FCT_MIXED = 1 };

/* Function families of fct_sample (synthetic workloads). */
enum {
  FCT_FAMILY_POLY = 0,          /* sum_m c_m T_m(x); params = c[N] (support order)        */
  FCT_FAMILY_GAUSSCOS = 1,      /* exp(-sum a_i x_i^2) cos(sum b_i x_i); params = a[D],b[D] */
  FCT_FAMILY_RATIONAL = 2,      /* 1/(1 + sum c_i x_i^2); params = c[D]                    */
  FCT_FAMILY_POLY_GAUSSCOS = 3, /* gausscos + poly; params = a[D], b[D], c[N]              */
  FCT_SAMPLE_FOLDED = 0x100     /* flag OR-ed into a polynomial family: evaluate the
                                   polynomial through its bins (see fct_sample)          */
};

typedef struct fct_plan_s* fct_plan;

#define FCT_GRID_EXTREMA 0
#define FCT_GRID_FIRST_KIND 1

typedef struct {
  int precision;      /* FCT_FP64: FP64 CG on the normal equations.  FCT_MIXED: FP32
                         inner solves between FP64 residual sweeps; if a sweep gains
                         less than one digit (ill-conditioned L-grid) or max_refine
                         sweeps pass, the solve continues in FP64 from the current x. */
  double tol;         /* stop when ||A^T r|| <= tol * ||A^T b|| (FP64 measure)           */
  int max_iter;       /* cap on CGLS iterations (FP64) / inner iterations per sweep     */
  double inner_tol;   /* FCT_MIXED: relative tolerance of each inner FP32 solve         */
  int max_refine;     /* FCT_MIXED: cap on FP64 refinement sweeps                       */
  int block_threads;  /* 0 = default (256).  Must be 128, 256 or 512 otherwise.         */
  int max_blocks;     /* 0 = all co-resident blocks; else cap on the solver's grid      */
  int coef_lanes;     /* 0 = auto; else 1, 2, 4, 8 or 16 threads per coefficient in A^T r */
  double timeout_s;   /* bound on any device-side wait (default 4 s)                    */
  int normal_matrix;  /* FCT_MIXED inner solve: 0 = auto, 1 = on, -1 = off.  On: the plan
                         stores W = A^T A (CSR, FP32) and the inner solve is CG on
                         W d = g in pipelined form (one team barrier per iteration
                         instead of two); auto turns it on when W has no more
                         nonzeros than A and A^T together (2 K N) and at most 8 M.   */
  int grid_kind;      /* FCT_GRID_EXTREMA (default): n extrema points cos(pi j/(n-1)),
                         interpolating DCT-I, unit alias entries.  FCT_GRID_FIRST_KIND:
                         the paper's own form, Eq. (chebyshev_grid) with n points
                         cos((j+1/2) pi/n), the 1/n DCT-II quadrature of Eq. (quad_1D)
                         and the signed entries 1, +-1/2, 0 of Eq. (aliasing_matrix_1d)
                         (Lemma lem:aliasing), multiplied over axes.  Single-point
                         axes sample the given node in both kinds.                  */
  int entries_per_lane; /* A p gather: 0 = auto (the fewest entries per lane, of 2, 4 or 8,
                         whose row units fit one wave of co-resident blocks: lowest
                         latency for one transform on the whole GPU); 2, 4 or 8 fixes
                         it.  Larger values mean fewer, longer units: better when
                         the plan runs on small teams (fct_execute_batch, serving),
                         where a block works through many units one after another. */
  int plan_build;     /* where fct_plan_create builds the alias tables: FCT_PLAN_BUILD_AUTO
                         (0, default) and FCT_PLAN_BUILD_DEVICE (2) on the GPU (fold,
                         stable radix sort by bin, compaction, row order: kernels),
                         FCT_PLAN_BUILD_HOST (1) in host C++.  Both give the same
                         tables bit for bit (fct_plan_tables).  The device build
                         needs transient scratch of about 110 bytes per entry (K N). */
  int tensor_dct;     /* DCT passes on the tensor cores (Algorithm 3's per-grid DCT as
                         BF16 digit-slice products with exact FP32 accumulation,
                         FP64-accurate): 0 = auto (grids whose longest axis has
                         64 to 1024 points), 1 = every grid with an active axis of at
                         most 1024 points, -1 = off (FP64 units only).  Used by
                         fct_execute, fct_execute_host and fct_plan_rhs; batches,
                         serving and fct_execute_noalloc transform every grid on
                         the FP64 units.                                              */
  int coef_split;     /* A^T q gather layout: 0 = auto (on for plans of 64 or more grids),
                         1 = grid-split: each gather warp takes 32 consecutive
                         coefficients of a chunk and every (block warps - 1)-th grid,
                         so its loads of the coefficient-major tables are coalesced and
                         its q reads fall in one grid's rows; the warps' partial sums
                         are added in warp order (coef_lanes is then unused).
                         -1 = lane-split: coef_lanes threads of one warp per
                         coefficient.  Both give results independent of the team
                         size; they differ from each other by rounding order only. */
  double kappa_max;   /* > 0: rank check (Algorithm 2's acceptance test, Sec. 3.3):
                         fct_plan_create estimates kappa(A) by 200 Lanczos steps of
                         fct_plan_condition from a fixed pseudo-random start and fails
                         with FCT_ERR_RANK when the estimate exceeds kappa_max or A
                         is rank-deficient.  0 (default) = no check.              */
} fct_options;

#define FCT_PLAN_BUILD_AUTO 0
#define FCT_PLAN_BUILD_HOST 1
#define FCT_PLAN_BUILD_DEVICE 2

typedef struct {
  int status;                 /* fct_status of this transform                        */
  int iterations;             /* CGLS iterations (FP64) or inner iterations (mixed)  */
  int refinements;            /* FP64 refinement sweeps (mixed path)                 */
  int reserved;
  double rel_normal_residual; /* ||A^T r|| / ||A^T b|| at exit, FP64                  */
  double gamma0;              /* ||A^T b||^2                                          */
} fct_report;

typedef struct {
  int64_t N;                /* support size (columns)                              */
  int64_t M;                /* samples over all grids                              */
  int64_t R;                /* nonempty bins over all grids (rows of A)            */
  int64_t nnz;              /* K*N                                                 */
  int32_t D, K;
  int32_t passes;           /* DCT passes (max active axes over grids)             */
  int32_t grid_blocks;      /* solver grid size used by fct_execute                */
  int32_t block_threads;
  int32_t coef_lanes;
  int64_t device_bytes;     /* tables + workspace held on the device               */
  int64_t normal_nnz;       /* nonzeros of W = A^T A when the plan stores it, else 0 */
  int64_t tensor_dct_grids; /* grids whose DCT runs on the tensor cores (fct_execute) */
  int32_t coef_split;       /* 1 when the A^T q gather is grid-split (fct_options.coef_split) */
  int32_t row_units;        /* A p gather units of the solver (each adds one partial sum) */
  int32_t wide_rows;        /* rows gathered by a whole block (the first row units)     */
  int32_t coef_chunks;      /* A^T q gather units of the solver                         */
  int32_t entries_per_lane; /* A p gather: entries per lane of a row unit (2, 4 or 8)   */
  int32_t kernel_variant;   /* solver kernel of fct_execute: 0 plain, 1 entry values staged
                               in shared memory, 2 deep gathers (twice the entries per
                               lane and round)                                          */
  int64_t tensor_dct_flops; /* BF16 tensor-core flops of the DCT passes per fct_execute
                               (36 digit-slice products of M 128 x N 64 x K 16 per tile
                               and K step); 0 without tensor-core grids              */
  double kappa_estimate;    /* the rank check's kappa(A) estimate (0 without the check) */
} fct_plan_info;

/* Fill *opt with defaults: FP64, tol 1e-13, max_iter 50000, inner_tol 1e-6,
 * max_refine 6, automatic launch shape, 4 s wait bound, normal matrix auto. */
void fct_default_options(fct_options* opt);

/* Thread-local message of the last failing call (never NULL). */
const char* fct_last_error(void);

/* Human-readable name of a status code. */
const char* fct_status_string(int status);

/*
 * Build a plan: the alias tables of every grid (Sec. 3.3, Algorithm 2 without
 * its condition-number loop; the L-grid is an input; built by kernels on the
 * current device unless opt->plan_build says host), the DCT-I matrices and the
 * solver workspace, all resident on the current device.  Every launch, copy,
 * scratch allocation (cudaMallocAsync) and release of the build is ordered on
 * a stream the call creates for itself, and only that stream is waited for,
 * so a plan can be built while other streams keep the device busy (e.g. a
 * running fct_server launch whose teams leave SMs free: a plan-cache miss
 * while serving).  The plan's tables and workspace are one cudaMalloc (two
 * with tensor-core grids).
 *   D in [1, 255]; N >= 1; support host uint16[N][D] (any multi-indices);
 *   K >= 1; sizes host int32[K][D], every n in [1, 4096], each grid's point count and
 *   the total M below 2^31, K*N below 2^31; nodes host double[K][D] in [-1,1]
 *   (read where n == 1; NULL means xi = 1); opt NULL = defaults.
 * Returns when the plan is ready.  Errors: FCT_ERR_INVALID_ARG, FCT_ERR_OOM,
 * FCT_ERR_CUDA, FCT_ERR_NO_DEVICE.  *out is NULL on failure.
 */
fct_status fct_plan_create(fct_plan* out, int D, int64_t N, const uint16_t* support,
                           int K, const int32_t* sizes, const double* nodes,
                           const fct_options* opt);

/*
 * A second handle on a plan's tables with its own solver workspace, so that
 * several transforms of the same shape can run at once (e.g. serving slots).
 * The tables stay on the device until the plan and all its clones are
 * destroyed.  Synchronous.  Errors: FCT_ERR_INVALID_ARG, FCT_ERR_OOM, FCT_ERR_CUDA.
 */
fct_status fct_plan_clone(fct_plan* out, fct_plan plan);

/* Plan geometry (host struct). */
fct_status fct_plan_get_info(fct_plan plan, fct_plan_info* info);

/* offsets host int64[K+1]: start of each grid's samples in the samples array. */
fct_status fct_grid_offsets(fct_plan plan, int64_t* offsets);

/*
 * Sample a synthetic function on the plan's L-grid (the "sample f" step of
 * Algorithm 3).  params host double[nparams] laid out per FCT_FAMILY_*;
 * samples device double[M].  Asynchronous on stream (params are staged
 * through plan-owned device memory before returning).
 * Polynomial families are evaluated term by term (M*N*D work) unless M*N
 * exceeds 4e10 or FCT_SAMPLE_FOLDED is set: then the coefficients are folded
 * into each grid's bins (the alias map) and the grid interpolant is evaluated
 * at the nodes, axis by axis (O(K N + M sum n) work).  The folded path uses
 * the plan's workspace: it must not overlap an execute on the same plan.
 */
fct_status fct_sample(fct_plan plan, int family, const double* params, int64_t nparams,
                      double* samples, void* stream);

/*
 * Execute Algorithm 3 on device-resident samples: per-grid DCT-I, bin gather,
 * CGLS (FP64 or mixed with FP64 refinement), coefficients out.
 *   samples device double[M] (read only); coeffs device double[N] (written).
 * One cooperative kernel launch on stream.  If rep != NULL the call waits for
 * the stream and fills *rep, returning rep->status; otherwise it returns after
 * the launch (status then only via a later fct_plan_last_report).
 */
fct_status fct_execute(fct_plan plan, const double* samples, double* coeffs, void* stream,
                       fct_report* rep);

/*
 * fct_execute with HOST buffers: copies samples host double[M] to the device,
 * executes, copies coeffs back to host double[N], and waits for the stream.
 * Pinned host memory gives asynchronous copies; pageable memory also works.
 */
fct_status fct_execute_host(fct_plan plan, const double* samples_host, double* coeffs_host,
                            void* stream, fct_report* rep);

/*
 * Solve B independent transforms in ONE persistent cooperative launch.  Teams
 * of blocks pull transforms from a device work queue; each transform's result
 * is bit-identical to its result alone under the same plan.
 *   plans host fct_plan[B] (distinct plans); samples host array of B device
 *   pointers; coeffs host array of B device pointers; reps host fct_report[B]
 *   or NULL (same waiting rule as fct_execute); team_blocks = blocks per team
 *   (0 = automatic).
 */
fct_status fct_execute_batch(int B, const fct_plan* plans, const double* const* samples,
                             double* const* coeffs, int team_blocks, void* stream,
                             fct_report* reps);

/*
 * A prepared batch: the job table of fct_execute_batch kept in device memory,
 * so that the launch itself needs nothing from the host.
 *   fct_batch_create: same arguments and rules as fct_execute_batch (the
 *     buffers and plans are bound to the batch; the caller keeps them alive
 *     and does not run those plans elsewhere while a launch of the batch is
 *     in flight).  Allocates the job table, the reports and a launch state,
 *     uploads the jobs and fixes the launch shape.  Synchronous.
 *   fct_batch_launch: one memset of the launch state and one cooperative
 *     launch (cudaLaunchKernelEx with the cooperative attribute) on stream;
 *     no host synchronisation, allocation or read of host memory, so the call
 *     can be recorded by stream capture into a CUDA graph and the graph
 *     replayed; every launch reads the samples as they are at its start and
 *     writes the coefficients and the device-side reports.
 *   fct_batch_reports: copies the B reports of the last completed launch into
 *     host fct_report[B] after waiting for stream; returns the worst status,
 *     or the launch's error code when a bounded device-side wait expired.
 *   fct_batch_destroy: waits for the device, frees the batch (not the plans).
 * Results are bit-identical to fct_execute_batch and to each transform alone.
 */
typedef struct fct_batch_s* fct_batch;
fct_status fct_batch_create(fct_batch* out, int B, const fct_plan* plans, const double* const* samples,
                            double* const* coeffs, int team_blocks);
fct_status fct_batch_launch(fct_batch batch, void* stream);
fct_status fct_batch_reports(fct_batch batch, void* stream, fct_report* reps);
fct_status fct_batch_destroy(fct_batch batch);

/*
 * fct_execute without any device allocation.  No counterpart in the paper: it
 * exists for callers that cannot allocate device memory when they solve, such
 * as code under a memory policy that forbids cudaMalloc after start-up (a
 * real-time loop, a fixed memory pool, a host runtime that owns the device
 * memory).  Such a caller creates its plans ahead of time; this call then runs
 * a plan with its solver workspace taken from one fixed 32 MiB array that the
 * library holds in every device's memory from load until process exit.  The
 * plan supplies only its read-only tables.  Same arguments and results as
 * fct_execute; no cudaMalloc, cudaFree or other allocating routine is called.
 *   - Plans whose workspace exceeds 32 MiB are rejected with
 *     FCT_ERR_INVALID_ARG (the message gives the bytes needed).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and keeps it for the life of the process; make
 *     that first call before any stream capture.  A process that resets the
 *     device (cudaDeviceReset) must not call this entry point afterwards.
 *   - All calls on a device share the array: calls that overlap on the GPU
 *     (different streams, or different plans at once) race and must not be
 *     issued.  The array keeps the last call's contents; the call clears what
 *     must start at zero itself.
 *   - The solve always runs on the team solver with its index tables staged in
 *     shared memory (fct_execute may also stage the entry values): results
 *     equal fct_execute's up to rounding.
 */
fct_status fct_execute_noalloc(fct_plan plan, const double* samples, double* coeffs, void* stream,
                               fct_report* rep);

/*
 * Serving with continuous batching.  A server owns one persistent launch whose
 * teams of blocks take jobs (plan, samples, coeffs) from a ring in host-mapped
 * memory as soon as they are submitted, so work submitted while other jobs run
 * overlaps with them on the device; a team that finishes a job takes the next
 * one.  Every team stays while any job runs; the launch ends once no job has
 * run for idle_timeout_s, and is started again by the next submit or by
 * polling an unclaimed job.
 *   fct_server_create: block_threads 0/128/256/512 (plans must match),
 *     team_blocks blocks per team (0 = 16), teams (0 = as many as fit), the
 *     launch occupies teams * team_blocks co-resident blocks while it runs;
 *     idle_timeout_s in (0, 1].
 *   fct_server_submit: samples device double[M], coeffs device double[N]; the
 *     caller keeps them alive and does not reuse the plan until the job is
 *     done (one job per plan at a time: a plan owns one workspace).  *ticket
 *     identifies the job; at most 4096 unfinished jobs (else FCT_ERR_OOM).
 *   fct_server_poll: *done = 1 and *rep filled once the job has finished.
 *   fct_server_wait: polls until done or timeout_s (FCT_ERR_TIMEOUT); returns
 *     the job's status.
 *   fct_server_destroy: asks the launch to stop, waits for it, frees the server.
 * Other kernels cannot start on the device while the launch holds all blocks:
 * size teams to leave room, or prepare inputs before submitting.
 */
typedef struct fct_server_s* fct_server;
fct_status fct_server_create(fct_server* out, int block_threads, int team_blocks, int teams,
                             double idle_timeout_s);
fct_status fct_server_submit(fct_server server, fct_plan plan, const double* samples, double* coeffs,
                             int64_t* ticket);
fct_status fct_server_poll(fct_server server, int64_t ticket, int* done, fct_report* rep);
fct_status fct_server_wait(fct_server server, int64_t ticket, double timeout_s, fct_report* rep);
fct_status fct_server_destroy(fct_server server);

/*
 * The alias operator alone (Eq. (L-grid_A_mat) with the rows of empty bins
 * dropped), from the plan's device tables in FP64:
 *   transpose = 0: out[R] = A in[N]   (rows in the plan's internal order);
 *   transpose = 1: out[N] = A^T in[R] (in[] in the internal row order).
 * in / out: device doubles; bins: host int64[R] or NULL, each row's sample
 * index (grid offset + row-major bin index).  For checks against a
 * reference.  Asynchronous on stream.
 */
fct_status fct_plan_apply(fct_plan plan, const double* in, double* out, int transpose, int64_t* bins, void* stream);

/*
 * The right-hand side alone (the first stage of fct_execute): every grid's
 * DCT of the samples (device double[M]), evaluated at the nonempty bins,
 * Eq. (main_linear_system)'s b = F f with the rows of empty bins dropped.
 *   b:    device double[R], in the plan's internal row order;
 *   bins: host int64[R] or NULL: for every row, the sample index of its bin
 *         (grid offset + row-major bin index), which identifies the row.
 * For checks of the DCT stage against a reference.  Synchronous.
 */
fct_status fct_plan_rhs(fct_plan plan, const double* samples, double* b, int64_t* bins, void* stream);

/*
 * The plan's alias tables, copied from the device into host buffers (any
 * pointer may be NULL to skip that table), rows in the plan's internal order:
 *   rowptr int32[R+1], col int32[K N], wcsr double[K N]: A's rows as CSR
 *     (one row per nonempty bin, columns ascending inside a row);
 *   crow int32[K N], wcm double[K N]: coefficient-major, [K][N], the row and
 *     value of column m's entry on grid l at l N + m;
 *   bins int64[R]: each row's sample index (grid offset + row-major bin).
 * For checking table builds against each other and against a reference.
 * Synchronous.  Errors: FCT_ERR_INVALID_ARG, FCT_ERR_CUDA.
 */
fct_status fct_plan_tables(fct_plan plan, int32_t* rowptr, int32_t* col, double* wcsr, int32_t* crow, double* wcm,
                           int64_t* bins);

/* Report of the plan's last execute (waits for stream). */
fct_status fct_plan_last_report(fct_plan plan, void* stream, fct_report* rep);

/*
 * Diagnostic of the bounded device waits: launches one block that waits at a
 * barrier meant for two, so the wait can only end by its time limit.
 * *status_out receives the status the device reported (FCT_ERR_TIMEOUT when
 * the limit works), *elapsed_s (may be NULL) the kernel's duration.
 * timeout_s in (0, 10].  Synchronous; allocates and frees a small state.
 */
fct_status fct_selftest_wait_timeout(double timeout_s, int* status_out, double* elapsed_s);

/*
 * Condition estimate for Algorithm 2 (Sec. 3.3: grids are appended while
 * kappa(A) exceeds a bound).  CG on A^T A is the Lanczos process: this runs
 * `iterations` FP64 CG iterations on A^T A z = start (start: device double[N],
 * a random vector reaches every eigenvector, including a null space of A;
 * work: device double[N], receives the iterate), reads back the CG
 * coefficients, builds the Lanczos tridiagonal and bisects its extreme
 * eigenvalues.  *lambda_min, *lambda_max estimate sigma_min^2 and
 * sigma_max^2 of A from inside; *kappa = sqrt(lambda_max / lambda_min) is a
 * lower bound on kappa(A) that tightens as iterations grow (the CG
 * coefficients come from FP64 inner products); *used = iterations recorded (fewer when the iteration breaks
 * down or the normal residual has fallen by 1e12, by which point the extreme
 * Ritz values have converged).  Outputs other than kappa may be NULL.
 * Synchronous.
 */
fct_status fct_plan_condition(fct_plan plan, const double* start, double* work, int iterations,
                              double* kappa, double* lambda_min, double* lambda_max, int* used, void* stream);

/*
 * Evaluate the expansion p(x) = sum_m coeffs[m] prod_i T_{m_i}(x_i)
 * (Eq. (chebyshev_expansion)) over the plan's support at npoints points, the
 * way the paper measures approximation error (at random points, Sec. 4).
 *   coeffs: device double[N], support order (fct_execute's output);
 *   points: device double[npoints][D], row-major, normally in [-1, 1]^D;
 *   values: device double[npoints].
 * T_k comes from the three-term recurrence up to the support's largest
 * degree.  npoints = 0 is a no-op.  Asynchronous on stream.
 */
fct_status fct_evaluate(fct_plan plan, const double* coeffs, int64_t npoints, const double* points, double* values,
                        void* stream);

/*
 * Measurement utility (no counterpart in the paper): time `rounds` crossings of
 * the library's team barrier by `blocks` co-resident blocks of block_threads
 * threads (128, 256 or 512) with no work in between; *us_per_barrier =
 * elapsed / rounds.  A CG iteration of the team solver crosses two barriers,
 * so this is the synchronisation floor of an iteration.  Every wait is
 * bounded (4 s).  Synchronous; allocates and frees its own small state.
 */
fct_status fct_measure_team_barrier(int blocks, int block_threads, int rounds, double* us_per_barrier);

/*
 * Measurement utilities (no counterpart in the paper): the on-chip roofs of a
 * solver whose working set stays in L2, measured on the current device.  Each
 * allocates and frees its own buffer, synchronises the device and changes no
 * device setting.
 *   fct_measure_l2: a buffer of `bytes` (1 to 96 MiB, so that it fits in L2)
 *     is read once to make it resident, then `passes` more times with 16-byte
 *     loads that bypass L1: *read_gbs = bytes read / time.  Then 8-byte loads
 *     at pseudo-random positions of the same buffer (the pattern of the alias
 *     gathers): *gather_gloads = 1e9 loads/s, *gather_sector_gbs = 32-byte
 *     sectors moved per second in GB/s (either may be NULL).
 *   fct_measure_fp64: independent FP64 fma chains in registers, `iters` fmas
 *     per chain: *tflops = 2 flops per fma / time.
 */
fct_status fct_measure_l2(int64_t bytes, int passes, double* read_gbs, double* gather_gloads,
                          double* gather_sector_gbs);
fct_status fct_measure_fp64(int iters, double* tflops);

/* Release a plan's device memory (synchronises the device first). NULL is OK. */
fct_status fct_destroy(fct_plan plan);

/*
 * Host-only alias tables (no device needed), for bit-exact checks:
 *   bin   host int32[K][N]: row-major bin of column m on grid l (the index of
 *         its one nonzero within grid l's full DCT output);
 *   crow  host int32[K][N]: global compressed row of that nonzero, rows
 *         numbered grid by grid, nonempty bins in ascending bin order;
 *   weight host double[K][N]: the entry, prod over n_i == 1 of T_{m_i}(xi_i)
 *         (first-kind grid: times the signed 1D entries of active axes; a
 *         degree with no entry on a grid gets bin index 0 on that axis and
 *         weight 0);
 *   *R_out: number of nonempty rows.  grid_kind: FCT_GRID_EXTREMA or
 *   FCT_GRID_FIRST_KIND (see fct_options).  Any output pointer may be NULL.
 */
fct_status fct_alias_tables_host(int D, int64_t N, const uint16_t* support, int K,
                                 const int32_t* sizes, const double* nodes, int grid_kind, int32_t* bin,
                                 int32_t* crow, double* weight, int64_t* R_out);

#ifdef __cplusplus
}
#endif
#endif /* FCT_H */
