/*
 * rlsq -- row-splitting ILU preconditioned sparse least squares on one GPU.
 *
 * Solves min_x || b - A x ||_2 for a sparse A (m x n, m > n, full column
 * rank): the problem of eq. (1.1) of Scott & Tuma, "Row-Splitting ILU
 * Preconditioners for Sparse Least-Squares Problems" (arXiv 2603.28642).
 *
 * The preconditioner is the paper's ILU row-splitting preconditioner:
 * a rectangular threshold-pivoted ILUP(p, tau) factorisation
 * P A D ~ [L1; L2] U (Algorithms 4-6, eq. 3.8) selects the square block A1,
 * and the remaining rows A2 enter through the algebraic correction with
 * Y = L2 L1^{-1} and S = I + Y Y^T (eq. 3.9, Algorithm 3, Lemma 3.1).
 * It is applied on the GPU once per iteration of LSMR as
 *     M^{-1} = D U^{-1} L1^{-1} K L1^{-T} U^{-T} D,
 *     K      = I - Y^T S^-1 Y   (S^ per the correction mode),
 * which with the exact S equals (A~^T A~)^{-1} for A~ = P^T [L1; L2] U D^{-1}
 * (the Woodbury form of Lemma 3.1).
 *
 * Conventions for every call:
 *  - Return value: RLSQ_OK (0), RLSQ_PENDING (> 0) or a negative RLSQ_ERR_*.
 *    On error, rlsq_last_error() gives a message (per calling thread).
 *    No call throws or aborts.
 *  - Index arrays: int64 row pointers, int32 column indices sorted strictly
 *    ascending within each row, float64 values.  The device copies use
 *    32-bit indices, so nnz(A) and nnz of each factor must be < 2^31.
 *  - ptr_mode RLSQ_HOST_PTRS: pointers are host memory; RLSQ_DEVICE_PTRS:
 *    device memory of the current CUDA device.  Inputs are always copied;
 *    the caller keeps ownership of every buffer it passes.
 *  - stream: a cudaStream_t (NULL = the legacy default stream).  Calls that
 *    take device pointers order their work on that stream; calls that take
 *    host pointers return after the result is in host memory.
 *  - Handles are owned by the caller until the matching destroy call.  A
 *    handle must not be used from two threads at the same time.
 */
#ifndef RLSQ_H
#define RLSQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RLSQ_OK 0
#define RLSQ_PENDING 1
#define RLSQ_ERR_ARG (-1)            /* null pointer, bad option value */
#define RLSQ_ERR_SHAPE (-2)          /* m <= n, n <= 0, or sizes over the 32-bit index limit */
#define RLSQ_ERR_CSR (-3)            /* bad row pointers, unsorted / duplicate / out-of-range columns, non-finite value */
#define RLSQ_ERR_RANK (-4)           /* A has an empty column (the paper removes null columns, Sec. 5.1) */
#define RLSQ_ERR_NOT_FACTORED (-5)   /* rlsq_factor has not succeeded on this handle */
#define RLSQ_ERR_OOM (-6)            /* device or host allocation failed */
#define RLSQ_ERR_BREAKDOWN (-7)      /* <s, M^{-1} s> <= 0 or not finite: the preconditioner is not positive */
#define RLSQ_ERR_MAXIT (-8)          /* iteration limit reached; x and info are still filled */
#define RLSQ_ERR_DEVICE_TIMEOUT (-9) /* a bounded device-side wait gave up (sync-free triangular solve) */
#define RLSQ_ERR_CUDA (-10)          /* a CUDA runtime call failed */
#define RLSQ_ERR_ADMISSION (-11)     /* server: request can never fit the memory budget */
#define RLSQ_ERR_NOT_FOUND (-12)     /* server: unknown ticket or matrix id */
#define RLSQ_ERR_NUMERIC (-13)       /* dense S not positive definite, NaN in b, ... */

/* ---- enums ---------------------------------------------------------------- */
#define RLSQ_HOST_PTRS 0
#define RLSQ_DEVICE_PTRS 1

/* correction modes: how Step 2 of Algorithm 3 (S w = u) is treated */
#define RLSQ_CORR_NONE 0   /* K = I: L1 and U only (no correction from A2) */
#define RLSQ_CORR_SI 1     /* S^ = I (Sec. 3.2, last paragraph); indefinite when ||Y|| > 1 */
#define RLSQ_CORR_CG 2     /* cg_steps CG iterations from zero on the implicit S (Sec. 3.2) */
#define RLSQ_CORR_DENSE 3  /* S assembled densely and inverted once (Sec. 3.2, Table 2 variant) */
#define RLSQ_CORR_AUTO 4   /* DENSE when m - n <= dense_cap, else CG */

#define RLSQ_PREC_FP64 0   /* preconditioner applied in float64 */
#define RLSQ_PREC_FP32 1   /* factors, D and the apply in float32; LSMR stays float64 */

#define RLSQ_TRSV_AUTO 0     /* choose per system (autotuned when autotune != 0) */
#define RLSQ_TRSV_LEVEL 1    /* one launch per level set */
#define RLSQ_TRSV_SYNCFREE 2 /* one launch, rows wait on the values they need (bounded waits) */
#define RLSQ_TRSV_COOP 3     /* one persistent launch, grid barrier between levels (bounded waits) */
#define RLSQ_TRSV_WAVE 4     /* one co-resident launch, a fixed row sequence per thread, rows wait on
                                their inputs and levels overlap (bounded waits) */
#define RLSQ_TRSV_BINNED 5   /* one persistent launch, grid barrier between level groups; within a
                                group rows are binned by length so that each lane gathers at most
                                four entries of its row per round (bounded waits) */

/* Krylov solvers of rlsq_solve */
#define RLSQ_SOLVER_LSMR 0  /* LSMR in x-space (the default) */
#define RLSQ_SOLVER_CGLS 1  /* preconditioned CGLS (Algorithm 1) with h = M^{-1} A^T r; no dense-row
                               problems */
#define RLSQ_SOLVER_CGLS_SPLIT 2 /* Algorithm 1 with h = Algorithm 3 applied to the residual split
                               (r1, r2) of r, the paper's combination of the preconditioner with
                               A^T (Sec. 3.2); no dense-row problems.  With exact factors and the
                               dense S^ it is one step; once entries are dropped h no longer
                               vanishes at the least-squares residual and the iteration stalls
                               above small tolerances (ends with RLSQ_ERR_MAXIT). */

/* triangular systems for rlsq_trsv */
#define RLSQ_SYS_L1 0   /* L1 x = b   (unit lower)      */
#define RLSQ_SYS_L1T 1  /* L1^T x = b (unit upper)      */
#define RLSQ_SYS_U 2    /* U x = b    (upper)           */
#define RLSQ_SYS_UT 3   /* U^T x = b  (lower)           */

/* factor parts for rlsq_get_factor */
#define RLSQ_PART_L1 0  /* strictly lower part of L1, n x n, rows = pivot positions */
#define RLSQ_PART_L2 1  /* L2, (m-n) x n, rows = A2 rows in ascending original id */
#define RLSQ_PART_U 2   /* strictly upper part of U, n x n */

typedef struct rlsq_problem_s *rlsq_problem;
typedef struct rlsq_server_s *rlsq_server;

/* Options of the set-up (Algorithm 4 inputs plus the correction choice). */
typedef struct {
    int32_t p;             /* max off-diagonal entries kept per column of L and of U; < 0: no limit */
    double tau;            /* absolute drop tolerance on the scaled matrix */
    double mu;             /* threshold pivoting parameter, 0 < mu <= 1 (Algorithm 5) */
    double small;          /* smallest admissible |U_jj| (Algorithm 6), > 0 */
    int32_t scale_columns; /* 1: prescale A to unit 2-norm columns (Sec. 5.1) */
    int32_t correction;    /* RLSQ_CORR_* */
    int32_t cg_steps;      /* CG iterations for RLSQ_CORR_CG, >= 1 */
    int64_t dense_cap;     /* RLSQ_CORR_AUTO uses DENSE when m - n <= dense_cap and the n x (m - n)
                              float64 buffer that forms S fits in 2 GiB, else CG */
    int32_t precision;     /* RLSQ_PREC_* */
    int32_t trsv_schedule; /* RLSQ_TRSV_* */
    int32_t autotune;      /* 1: time candidate kernel mappings on this matrix (lanes of the sparse
                              products, triangular-solve schedules); 2: only the lanes of the
                              sparse products A, A^T, L2, L2^T (all the batched and served forms
                              use); 0: heuristics */
    int64_t dense_row_min; /* rows of A with at least this many nonzeros are kept as dense
                              rows and multiplied by a dense-row GEMV block; 0 = automatic,
                              < 0 = never */
    int32_t host_threads;  /* host threads of the set-up: the ILUP column loop (pipelined over
                              columns, the same factor bit for bit for any count) and the dense
                              S; <= 0 = the CPUs the process may run on (the ILUP takes at most 16, and
                              fewer where its per-thread arrays, 16 bytes per row of A, would
                              pass 2 GiB); set-ups running at the same time should each get a
                              share of the CPUs */
    int32_t level_merge;   /* levels fused per group in the triangular solves: 1 = none,
                              k > 1 = groups of k levels (same-group dependencies are
                              substituted on the host), 0 = chosen per system by a
                              cost model (per level and per stored entry) among
                              k = 1..4 and groups grown level by level (a level
                              joins while the fill it adds costs less than a level) */
    int32_t trsv_rows;     /* RLSQ_TRSV_SYNCFREE without autotuning: 0 = blocks take chunks of
                              rows from the ticket counter; 1, 2 or 4 = warps take chunks and
                              each group of lanes solves that many rows, loading all their
                              structure before it waits on an unknown */
    double cg_tol;         /* RLSQ_CORR_CG: stop the CG iteration on S after the step that brings
                              ||r_j|| to at most cg_tol ||r_0|| (cg_steps is then the largest
                              count); 0 = always cg_steps steps.  Single-problem solves only:
                              rlsq_batch_solve and rlsq_server_register refuse it (ARG) */
    int32_t dense_host;    /* RLSQ_CORR_DENSE: 0 = form S^{-1} on the GPU (Z = L1^{-T} L2^T by a
                              multi-right-hand-side solve, S = I + Z^T Z, Cholesky, inverse; Z
                              must fit in 80% of the free device memory: OOM otherwise);
                              1 = on the host threads, keeping S^{-1} (and Z within 2 GiB) so
                              that rlsq_add_rows / rlsq_remove_rows update it by block
                              inversion instead of forming it again */
    int32_t sliced;        /* layout of the A, A^T, L2 and L2^T products: 1 = sliced (one lane
                              per row; rows sorted by length within windows of 1024, slices of
                              32 rows stored column-major), 0 = CSR with G lanes per row,
                              -1 (default) = the autotuner times both per product (CSR without
                              autotuning; the sliced copies are then not built).  The sums are the
                              same in both layouts when G = 1; the batched and served forms use CSR */
} rlsq_factor_opts;

/* Options of a solve. */
typedef struct {
    double atol;         /* stop when ||A^T r|| / (||A||_2 ||r||) < atol */
    int32_t maxit;       /* iteration limit */
    int32_t ptr_mode;    /* RLSQ_HOST_PTRS or RLSQ_DEVICE_PTRS for b and x */
    void *stream;        /* cudaStream_t */
    int32_t check_every; /* iterations per captured CUDA graph between host checks (>= 1) */
    int32_t solver;      /* RLSQ_SOLVER_*; the same stopping test for every solver (the CGLS forms use
                            the recurrence residual of Algorithm 1) */
} rlsq_solve_opts;

/* Result and statistics of a factorisation / solve. */
typedef struct {
    int32_t status;        /* RLSQ_OK, RLSQ_ERR_MAXIT, RLSQ_ERR_BREAKDOWN, ... */
    int32_t iterations;    /* LSMR iterations k of the returned x_k */
    double ratio;          /* ||A^T r_k|| / (||A||_2 ||r_k||) of the returned x_k */
    double rnorm;          /* ||r_k|| */
    double arnorm;         /* ||A^T r_k|| */
    double anorm;          /* ||A||_2 estimate (50 power iterations on A^T A) */
    double factor_seconds; /* host set-up + upload */
    double solve_seconds;  /* wall time of the solve call */
    int64_t m, n, nnz_A, nnz_L1, nnz_L2, nnz_U, nmod, n_dense_rows;
    int32_t levels_L1, levels_L1t, levels_U, levels_Ut;
    int32_t correction;    /* the resolved mode */
    int32_t precision;
    double bytes_per_iter; /* algorithmic HBM bytes of one LSMR iteration */
    int32_t solve_levels[4]; /* levels the GPU walks per system after fusing (RLSQ_SYS_* order) */
    int32_t level_merge[4];  /* fused levels per group, per system (groups chosen level by level:
                                the largest group) */
    int32_t trsv_schedule[4]; /* RLSQ_TRSV_* each system runs with (after autotuning) */
    double ilup_seconds;   /* host ILUP (Algorithms 4-6), split, transposes and level sets of the
                              factorisation in use (part of factor_seconds) */
    int32_t ilup_threads;  /* threads of its column loop */
    int64_t solve_entries[4]; /* stored entries the GPU reads per solve, per system, after level fusion
                                 (substituted and right-hand-side terms; the diagonal of U, U^T
                                 included); bytes_per_iter counts the factor's own entries */
    int32_t sliced_products;  /* products running in the sliced layout: 1 = A, 2 = A^T, 4 = L2,
                                 8 = L2^T (bits) */
} rlsq_info;

/* Server options and statistics (continuous batching of right-hand sides). */
typedef struct {
    int64_t hbm_budget_bytes; /* admission limit on resident per-request state */
    int32_t max_slots;        /* concurrent requests on the device */
    double atol;
    int32_t maxit;
} rlsq_server_opts;

typedef struct {
    int64_t submitted, completed, queued, active;
    double p50_ms, p99_ms, mean_ms;  /* submit -> result available */
    double solves_per_s;             /* completed / (last completion - first submit) */
    int64_t ticks;                   /* batched iterations run */
    int64_t peak_bytes;              /* largest admitted state footprint */
    double tick_ms;                  /* mean wall time of a tick (admission, launch, results) */
    double tick_device_ms;           /* mean part of it from graph launch to the device finishing */
} rlsq_server_stats;

/* ---- defaults -------------------------------------------------------------- */
/* p = 10, tau = 1e-2, mu = 0.1, small = 1e-10 (the paper's values, Sec. 5.2),
   scale_columns = 1, correction = AUTO, cg_steps = 2, dense_cap = 1024,
   precision = FP64, trsv_schedule = AUTO, autotune = 0, dense_row_min = 0,
   level_merge = 0. */
void rlsq_factor_opts_default(rlsq_factor_opts *opts);
/* atol = 1e-8, maxit = 2000, host pointers, default stream, check_every = 8, LSMR */
void rlsq_solve_opts_default(rlsq_solve_opts *opts);

/* ---- problem handle ------------------------------------------------------- */

/* Validate and copy A (CSR, m x n, m > n) and upload it (CSR, plus a CSC copy
   used for the deterministic A^T products).  ||A||_2 is estimated here.
   Errors: ARG, SHAPE, CSR, RANK, OOM, CUDA. */
int rlsq_create(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                const double *vals, int32_t ptr_mode, void *stream, rlsq_problem *out);

/* Host set-up of the preconditioner (Algorithms 4-6, split, level sets,
   correction set-up) and upload of the factors.  May be called again with
   other options.  Errors: ARG, NUMERIC (dense S not SPD), OOM, CUDA. */
int rlsq_factor(rlsq_problem h, const rlsq_factor_opts *opts);

/* Preconditioned LSMR from x0 = 0.  b has length m, x (output) length n,
   both in ptr_mode memory.  info may be NULL.  Returns OK, MAXIT (x holds
   the last iterate), BREAKDOWN, DEVICE_TIMEOUT, NOT_FACTORED, CUDA. */
int rlsq_solve(rlsq_problem h, const double *b, double *x, const rlsq_solve_opts *opts,
               rlsq_info *info);

/* Unpreconditioned LSMR (M = I) with the same kernels and stopping rule:
   the baseline the preconditioner is compared with. */
int rlsq_solve_plain(rlsq_problem h, const double *b, double *x, const rlsq_solve_opts *opts,
                     rlsq_info *info);

/* Solve `count` independent problems together: every LSMR iteration advances
   all unfinished problems with one batched launch sequence (one captured
   graph per iteration).  hs[i] must be factored; bs[i] (length m_i) and xs[i]
   (length n_i) follow opts->ptr_mode.  infos may be NULL.  Returns OK when
   every problem converged, otherwise the first non-OK status; per-problem
   status is in infos[i].status. */
int rlsq_batch_solve(rlsq_problem const *hs, const double *const *bs, double *const *xs,
                     int32_t count, const rlsq_solve_opts *opts, rlsq_info *infos);

/* One application t = M^{-1} s (both length n, ptr_mode memory). */
int rlsq_apply(rlsq_problem h, const double *s, double *t, int32_t ptr_mode, void *stream);

/* Algorithm 3 (Sec. 3.2) fed the residual split of r: r1 = r[prow] (the rows
   of A1), r2 = r[a2rows] (the rows of A2), u = r2 - L2 L1^{-1} r1, S^ w = u
   (the handle's correction: none, S^ = I, CG steps or dense), y = r1 +
   L1^{-T} L2^T w, L1 v = y, U h = v, t = D h.  r has length m (the rows in
   the order given to rlsq_create), t length n; both follow ptr_mode (device
   pointers are ordered after `stream`, the call returns when t is written).
   The factor's apply precision is used.  RLSQ_ERR_ARG for dense-row problems,
   RLSQ_ERR_NOT_FACTORED before rlsq_factor, RLSQ_ERR_DEVICE_TIMEOUT when a
   bounded wait of a triangular solve ran out. */
int rlsq_apply_residual(rlsq_problem h, const double *r, double *t, int32_t ptr_mode, void *stream);

/* y = A x (trans = 0; x length n, y length m) or y = A^T x (trans = 1). */
int rlsq_matvec(rlsq_problem h, int32_t trans, const double *x, double *y, int32_t ptr_mode,
                void *stream);

/* Solve one of the triangular systems RLSQ_SYS_* with the uploaded factor
   (in the factor's apply precision; float64 in and out). */
int rlsq_trsv(rlsq_problem h, int32_t which, const double *b, double *x, int32_t ptr_mode,
              void *stream);

/* Statistics of the current factorisation (iterations fields are zero). */
int rlsq_get_info(rlsq_problem h, rlsq_info *info);

/* Copy out the factor structure (host memory).  prow: n pivot rows in pivot
   order; a2rows: the m - n remaining rows ascending; d: n column scales;
   any pointer may be NULL. */
int rlsq_get_split(rlsq_problem h, int32_t *prow, int32_t *a2rows, double *d, double *udiag);
/* part RLSQ_PART_*: CSR arrays sized from rlsq_get_info (rows + 1, nnz, nnz). */
int rlsq_get_factor(rlsq_problem h, int32_t part, int64_t *ptr, int32_t *idx, double *val);
/* Level of every row of system RLSQ_SYS_* (length n). */
int rlsq_get_levels(rlsq_problem h, int32_t which, int32_t *level);

/* Sec. 3.4 on a factored handle (no counterpart in the paper beyond that
   section): add k rows (host CSR over the n columns; they join A2 with ids
   m .. m+k-1 and get L2 rows l with l U = a D, dropped by the factor's rule),
   or remove rows of A2 (ids ascending and distinct; the rest are renumbered in
   order).  L1 and U are kept; A's device copy, the m-sized vectors and the
   device factor are rebuilt with the handle's factor options (autotuning
   again if it was on).  b of later solves has the new m.  Errors: ARG (a
   pivot row cannot be removed: refactorise; the handle is registered with a
   live server), CSR, SHAPE (sizes past 2^31; a removal that would leave no
   row of A2, i.e. m <= n), NOT_FACTORED, OOM, CUDA. */
int rlsq_add_rows(rlsq_problem h, int64_t k, const int64_t *rowptr, const int32_t *colidx, const double *vals);
int rlsq_remove_rows(rlsq_problem h, int64_t k, const int32_t *ids);
/* Free the handle and its device memory.  A handle registered with a live
   server is left in place and the last error set (rlsq_server_register). */
void rlsq_destroy(rlsq_problem h);

/* ---- continuous-batching server ------------------------------------------ */

/* Create a server with its own scheduler thread and CUDA stream. */
int rlsq_server_create(const rlsq_server_opts *opts, rlsq_server *out);
/* Make a factored problem available to requests; the problem must outlive
   the server.  Until the server is destroyed, rlsq_factor, rlsq_add_rows and
   rlsq_remove_rows on the problem fail with ARG and rlsq_destroy leaves it in
   place (setting the last error).  Errors: ARG, NOT_FACTORED, ADMISSION (state
   larger than the whole budget). */
int rlsq_server_register(rlsq_server s, rlsq_problem h, int32_t *matrix_id);
/* Queue a solve with right-hand side b (host memory, length m of the matrix;
   copied before return, never blocks on the device).  ticket identifies the
   request. */
int rlsq_server_submit(rlsq_server s, int32_t matrix_id, const double *b, int64_t *ticket);
/* RLSQ_PENDING while queued or running; otherwise writes x (host, length n)
   and info (may be NULL) and returns the solve's status; a ticket can be
   collected once. */
int rlsq_server_poll(rlsq_server s, int64_t ticket, double *x, rlsq_info *info);
int rlsq_server_get_stats(rlsq_server s, rlsq_server_stats *stats);
void rlsq_server_destroy(rlsq_server s);

/* ---- measurement ---------------------------------------------------------
 * Per-iteration timing of the preconditioned LSMR loop on device-resident
 * data (no copies in the timed region).  After `warmup` untimed iterations,
 * `iters` iterations are replayed from the captured graph and timed with
 * CUDA events on the library's stream (total_ms).  Then one more iteration
 * is run kernel by kernel with an event pair around every launch; launches
 * are attributed to the RLSQ_KCLASS_* classes with the algorithmic HBM bytes
 * each class moves (every stored nonzero and vector element once).  The
 * solve runs with atol = 0 so it never stops early; if it ends anyway
 * (breakdown), status says so.  plain != 0 profiles the unpreconditioned
 * loop. */
#define RLSQ_KCLASS_SPMV 0    /* A v^ and A x with the LSMR epilogue */
#define RLSQ_KCLASS_SPMVT 1   /* A^T u and A^T r */
#define RLSQ_KCLASS_TRSV_L1 2
#define RLSQ_KCLASS_TRSV_L1T 3
#define RLSQ_KCLASS_TRSV_U 4
#define RLSQ_KCLASS_TRSV_UT 5
#define RLSQ_KCLASS_L2 6      /* products with L2 (incl. CG's S p) */
#define RLSQ_KCLASS_L2T 7     /* products with L2^T */
#define RLSQ_KCLASS_VEC 8     /* CG vector updates, dense S^{-1} GEMV */
#define RLSQ_KCLASS_FINISH 9  /* t = D g, <t, s>, rotations */
#define RLSQ_KCLASS_UPDATE 10 /* h-bar, x, h */
#define RLSQ_KCLASS_DENSE 11  /* dense-row GEMV block */
#define RLSQ_KCLASS_COUNT 12
typedef struct {
    int32_t status;
    int32_t iters;
    double total_ms;                       /* graph replay of `iters` iterations */
    double class_ms[RLSQ_KCLASS_COUNT];    /* one eager iteration, per class */
    int32_t class_launches[RLSQ_KCLASS_COUNT];
    double class_bytes[RLSQ_KCLASS_COUNT]; /* algorithmic bytes per iteration */
    double bytes_per_iter;
} rlsq_profile_out;
int rlsq_profile(rlsq_problem h, const double *b, int32_t warmup, int32_t iters, int32_t plain,
                 rlsq_profile_out *out);

/* ---- allocation-free triangular solve ---------------------------------------
 * The paper has no counterpart to this call; it exists for callers that must
 * not allocate device memory while they run -- a latency-critical serving
 * loop, where a cudaMalloc can stall the whole device, or a process whose
 * free device memory is already held by another allocator.
 *
 * rlsq_trsv_noalloc solves the triangular system `which` (RLSQ_SYS_*) of a
 * problem factored with RLSQ_PREC_FP64, like rlsq_trsv, with the sync-free
 * kernel.  b (input) and x (output) are caller-owned DEVICE arrays of length n
 * on the problem's device; the work is ordered on `stream` and the call
 * returns after it finished.  It calls no cudaMalloc / cudaFree: the solve's
 * working memory (ready flags, ticket counter, error word) lives in one
 * statically sized device array of RLSQ_NOALLOC_MAX_ROWS + 128 32-bit words
 * (8 MiB + 512 B) that every GPU which loads the library keeps until the
 * process exits.
 *  - n > RLSQ_NOALLOC_MAX_ROWS is rejected with RLSQ_ERR_SHAPE (nothing runs).
 *  - The first call on a device (and the first after a device reset) looks
 *    up the array's device address (cudaGetSymbolAddress) with that device
 *    current; make that first call before any stream capture.
 *  - The call is synchronous: it waits on `stream` for the solve to finish
 *    and reads the error word back before it returns.
 *  - Every call reuses the same array and clears what must start at zero;
 *    calls that overlap on the GPU (other streams, other threads, other
 *    problems) race on it and must be serialised by the caller.
 *  - Errors: ARG (null pointer, bad id, float32 factor, other device),
 *    NOT_FACTORED, SHAPE, DEVICE_TIMEOUT, CUDA. */
#define RLSQ_NOALLOC_MAX_ROWS 2097152
int rlsq_trsv_noalloc(rlsq_problem h, int32_t which, const double *b, double *x, void *stream);

/* ---- host-only set-up (no GPU needed) -------------------------------------
 * The row-selecting rectangular ILU set-up that rlsq_factor runs, callable on
 * its own: column scaling (Sec. 5.1), ILUP(p, tau) with threshold pivoting
 * (Algorithms 4-6), the split P A D ~ [L1; L2] U (eq. 3.8) and the level
 * sets of L1, L1^T, U, U^T.  Inputs are host CSR arrays (copied); only
 * opts->p, tau, mu, small, scale_columns and host_threads are used.  Errors:
 * ARG, SHAPE, CSR, RANK. */
typedef struct rlsq_setup_s *rlsq_setup;
int rlsq_setup_create(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                      const double *vals, const rlsq_factor_opts *opts, rlsq_setup *out);
/* Host threads the ILUP column loop of an m x n set-up takes when
   host_threads = requested (the rule of rlsq_factor_opts.host_threads; the
   factor does not depend on it).  Never fails; returns >= 1. */
int32_t rlsq_setup_threads(int32_t requested, int64_t m, int64_t n);
/* sizes[0..7] = nnz(L1 strict), nnz(L2), nnz(U strict), nmod,
   levels of L1, L1^T, U, U^T */
int rlsq_setup_sizes(rlsq_setup s, int64_t *sizes);
/* The same arrays, layouts and errors as rlsq_get_split, rlsq_get_factor
   (sizes from rlsq_setup_sizes) and rlsq_get_levels of a factored handle. */
int rlsq_setup_split(rlsq_setup s, int32_t *prow, int32_t *a2rows, double *d, double *udiag);
int rlsq_setup_factor(rlsq_setup s, int32_t part, int64_t *ptr, int32_t *idx, double *val);
int rlsq_setup_levels(rlsq_setup s, int32_t which, int32_t *level);
/* Level fusion of triangular system `which` (RLSQ_SYS_*) as rlsq_factor does
   it (no counterpart in the paper): k >= 1 fuses groups of k consecutive
   levels, k = 0 grows groups level by level under the library's float64 cost
   model.  Inside a group the dependencies on rows of the same group are
   substituted, so row i reads x_i = (rhs_i + sum_R c rhs_j - sum_T c x_j) / d_i
   (d = 1 for L1, L1^T; U's diagonal for U, U^T) with every T dependency in an
   earlier group.  The result stays in the handle until the next call.
   out[0..3] = stored entries of T, of R, levels of T, levels in the largest
   group.  Errors: ARG. */
int rlsq_setup_fuse(rlsq_setup s, int32_t which, int32_t k, int64_t *out);
/* CSR of the last fused system, rows and columns = unknown ids: part 0 = T,
   1 = R; ptr has n + 1 entries, idx / val the counts rlsq_setup_fuse gave.
   Errors: ARG (bad part, no fused system). */
int rlsq_setup_fused(rlsq_setup s, int32_t part, int64_t *ptr, int32_t *idx, double *val);
/* Sec. 3.4, adding rows: k rows (host CSR over the n columns, the user's
   values) join A2 with ids m .. m+k-1; each gets the L2 row l solving
   l U = a D with L1, U, D and the pivots unchanged, dropped by the factor's
   (tau, p) rule.  Later rlsq_setup_* getters see the updated factor
   (rlsq_setup_sizes, _split with the new m, _factor).  Errors: ARG, CSR, SHAPE. */
int rlsq_setup_add_rows(rlsq_setup s, int64_t k, const int64_t *rowptr, const int32_t *colidx,
                        const double *vals);
/* Sec. 3.4, removing rows of A2: ids ascending and distinct; their L2 rows go
   and the remaining rows are renumbered in order (ids above a removed row move
   down).  A pivot row cannot be removed this way: ARG (refactorise).  At
   least one row of A2 must remain (m > n): SHAPE otherwise. */
int rlsq_setup_remove_rows(rlsq_setup s, int64_t k, const int32_t *ids);
/* S^{-1} of the dense correction (S = I + Z^T Z, Z = L1^{-T} L2^T, eq. 3.9;
   Lemma 3.1), row-major (m-n) x (m-n) into out.  Formed (through the Cholesky
   factor of S) on the first call or when recompute != 0; after that the
   handle keeps it, with Z while Z (n x (m-n) float64) fits in 2 GiB, and
   rlsq_setup_add_rows / rlsq_setup_remove_rows update it by block inversion
   through the Schur complement (Sec. 3.4): O(n (m-n) + (m-n)^2) per added row,
   O((m-n)^2) per removed row, instead of forming it again (which they do
   where the update would lose more than 4 digits, or without Z).  Errors:
   ARG, NUMERIC (S not positive definite). */
int rlsq_setup_schur_inverse(rlsq_setup s, int32_t recompute, double *out);
void rlsq_setup_destroy(rlsq_setup s);

/* Message of the last error on this thread ("" if none). */
const char *rlsq_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RLSQ_H */
