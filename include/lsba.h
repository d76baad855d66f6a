/*
 * lsba.h -- C ABI of the GB300 (sm_103a) low-synchronization block Arnoldi
 * solver for A X = B: restarted, adaptively restarted BFOM / BGMRES.
 *
 * Method: K. Lund, "Adaptively restarted block Krylov subspace methods with
 * low-synchronization skeletons" (arXiv 2208.09899).
 *   - problem A X = B, A n x n sparse, B n x s, s << n            (Sec. 2, Eq. (1))
 *   - classical block inner product <X,Y> = X^T Y                  (Table 1)
 *   - skeletons: BCGS (Sec. 3.1), BCGS-PIP (Alg. 3), BMGS-CWY and
 *     BMGS-ICWY (Alg. 6), BCGSI+LS (Alg. 7); muscle CholQR        (Sec. 2.3, Sec. 5)
 *   - modified BFOM / BGMRES solution and cospatial residual      (Eq. (7), Thm. 1, Eq. (9))
 *   - static restarts (Sec. 2.4.2) with adaptive restarting on a
 *     Cholesky NaN-flag                                            (Sec. 4)
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers on the handle's device; h_* are
 *     host pointers.  The caller owns every buffer it passes and keeps it alive
 *     until the call returns.
 *   - Block vectors are n x s, FP64, row-major (the s values of a row are
 *     contiguous; a C-contiguous (n, s) array).  s must be 1..32.
 *   - CSR matrices are 0-based, int32 row pointers and column indices (columns
 *     sorted within a row), FP64 values; nnz < 2^31.
 *   - Every call is ordered on the handle's CUDA stream and returns when its
 *     results are complete (blocking).  One handle per host thread.
 *   - Errors are returned as lsba_status codes, never thrown; no call aborts
 *     the process.  A failed CUDA call leaves the handle usable only for
 *     lsba_destroy.
 */
#ifndef LSBA_H
#define LSBA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsba_ctx* lsba_handle;

/* Status codes. */
enum {
  LSBA_OK = 0,
  LSBA_NOT_CONVERGED = 1,   /* X holds the last iterate                        */
  LSBA_BREAKDOWN = 2,       /* CholQR of B flagged (numerically rank-deficient B) */
  LSBA_INVALID_ARG = 3,
  LSBA_OUT_OF_MEMORY = 4,
  LSBA_CUDA_ERROR = 5,
  LSBA_DEVICE_TIMEOUT = 6   /* a kernel's bounded wait (mbarrier, one second at
                               most) gave up; the kernel recorded it and returned */
};

/* Block Arnoldi skeletons (names as in the paper, Sec. 3). */
typedef enum {
  LSBA_BCGS = 0,            /* Sec. 3.1, 2 syncs per step                     */
  LSBA_BCGS_PIP = 1,        /* Alg. 3, 1 sync per step                        */
  LSBA_BCGSI_LS = 2,        /* Alg. 7, 1 sync per step, lagged normalization  */
  LSBA_BMGS_ICWY = 3,       /* Alg. 6 (inverse compact WY branch)             */
  LSBA_BMGS_CWY = 4,        /* Alg. 6 (compact WY branch)                     */
  LSBA_BMGS = 5,            /* Alg. 2, k + 1 syncs in step k (the comparator)  */
  LSBA_BCGS_PIO = 6,        /* Alg. 4, 2 syncs per step (muscle CholQR)        */
  LSBA_BMGS_SVL = 7,        /* Alg. 5 (Schreiber-Van Loan), 3 syncs per step    */
  LSBA_BMGS_LTS = 8         /* Alg. 5 (lower triangular solve), 3 syncs per step */
} lsba_skeleton;

/* Low-rank modification of BFOM (Sec. 2.4.1, Eq. (7)). */
enum { LSBA_FOM = 0, LSBA_GMRES = 1 };

/* CSR matrix; all pointers are device pointers. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t* d_rowptr;  /* n+1 */
  const int32_t* d_colidx;  /* nnz */
  const double* d_vals;     /* nnz */
} lsba_csr;

/* Solver options.  lsba_default_options() fills the defaults shown. */
typedef struct {
  int32_t modification;          /* LSBA_GMRES (default) or LSBA_FOM                    */
  int32_t max_restarts;          /* 50: at most max_restarts+1 cycles                   */
  int32_t adaptive_restart;      /* 1: on a Cholesky flag shrink m and restart (Sec. 4);
                                    0: a flag ends the solve (NOT_CONVERGED)            */
  int32_t verify_true_residual;  /* 1: confirm convergence with ||B - A X||_F/||B||_F;
                                    if above tol, restart from B - A X                  */
  int32_t record_history;        /* 1: keep per-step estimates, the first cycle's Gram
                                    outputs and Hessenberg matrix (lsba_get_history)    */
  int32_t inject_flag_cycle;     /* test hook: force the Cholesky flag while completing */
  int32_t inject_flag_relation;  /* relation inject_flag_relation of cycle
                                    inject_flag_cycle (1-based); -1 disables            */
  int32_t profile;               /* 1: time every kernel launch with CUDA events on the
                                    handle's stream (lsba_get_profile)                  */
  int32_t precision;             /* arithmetic of the SpMM, Gram and update passes:
                                    LSBA_PREC_DF: double-float (hi + lo FP32 pairs, 48
                                    significand bits, 8 bytes per entry) on the FP32
                                    pipes; LSBA_PREC_FP64: native FP64 (DFMA);
                                    LSBA_PREC_AUTO (default): for BCGSI+LS and
                                    BMGS-CWY/ICWY FP64 on the tensor cores where
                                    those passes take the shape (s = 8, m <= 22,
                                    tensor_cores != 0), else DF; FP64 for BCGS and
                                    BCGS-PIP, whose O(eps) kappa^2 loss of
                                    orthogonality (Table 2) amplifies the 2^-48
                                    representation error.  The small s x s / ks x s
                                    kernels are FP64 in all modes.  DF takes every
                                    s <= 32 and m.  FP64 runs the Gram and the
                                    update of the lagged skeletons, BCGS-PIP,
                                    BCGS-PIO and BCGS at s = 8, m <= 22 as exact
                                    products of 8-bit digits on
                                    the tensor cores (53 bits per value relative to
                                    its 128-row tile and column, FP64
                                    accumulation; tensor_cores = 0 turns this off).
                                    LSBA_PREC_FP32_IR: FP64 iterative refinement
                                    (residual B - A X and X += D in FP64) around an
                                    FP32 inner solve of A D = R (FP32 SpMM, Gram and
                                    update with FP32 accumulation; FP64 Cholesky and
                                    least squares); s must be 4, 8 or 16.            */
  int32_t ir_max_outer;          /* FP32_IR: at most this many refinement steps (10)   */
  double ir_inner_tol;           /* FP32_IR: relative residual of each inner solve (1e-5) */
  int32_t cuda_graphs;           /* 1 (default): a restart cycle whose launch sequence
                                    (matrix, block buffers, basis size, start mode,
                                    skeleton, precision, workspace) is seen a second
                                    time is captured into a CUDA graph, and later
                                    occurrences replay it (same kernels, same
                                    results); 0: every launch is issued directly.
                                    Off while profile = 1.                            */
  int32_t tensor_cores;          /* 1 (default): the tensor-core digit kernels run
                                    where they are faster: in FP64 the Gram and
                                    update of the lagged skeletons, BCGS-PIP,
                                    BCGS-PIO and BCGS at s = 8, m <= 22;
                                    in DF the passes of those skeletons at s = 8 and
                                    other Grams with b s = 16, a s >= 160,
                                    a s + b s <= 256 (exact digit products, 48-bit
                                    accuracy); 2: also every DF pass whose shape the
                                    kernel allows; 0: FP64 and FP32-pipe kernels
                                    only.                                              */
  int32_t inner_product;         /* block inner product (Sec. 2.2, Table 1):
                                    LSBA_IP_CLASSICAL (default): <X, Y> = X^T Y, muscle
                                    CholQR; LSBA_IP_GLOBAL: <X, Y> = tr(X^T Y)/s I_s,
                                    muscle the global scaling quotient ||X||_F/sqrt(s)
                                    I_s.  Every skeleton takes either; the Gram passes
                                    are the same, and each s x s block of their result
                                    is replaced by its trace / s times I_s.            */
  int32_t muscle;                /* muscle of BMGS-SVL / BMGS-LTS under the classical
                                    product: LSBA_MUSCLE_CHOLQR (default) or
                                    LSBA_MUSCLE_COLUMN, the column muscles MGS-SVL /
                                    MGS-LTS (3s - 2 syncs per call, Sec. 5 list of
                                    muscles); any other skeleton or the global
                                    product with LSBA_MUSCLE_COLUMN is
                                    LSBA_INVALID_ARG.                                  */
  int32_t inject_stall;          /* test hook (0 in normal use): 1 makes the start
                                    kernel of the first cycle wait, boundedly, on an
                                    mbarrier that nothing arrives at; the wait gives
                                    up after one second, the kernel records the
                                    error, the remaining kernels of the cycle skip
                                    their work and the solve returns
                                    LSBA_DEVICE_TIMEOUT (X undefined).  The handle
                                    stays usable.                                      */
} lsba_options;

enum { LSBA_PREC_FP64 = 0, LSBA_PREC_DF = 1, LSBA_PREC_AUTO = 2, LSBA_PREC_FP32_IR = 3 };
enum { LSBA_IP_CLASSICAL = 0, LSBA_IP_GLOBAL = 1 };
enum { LSBA_MUSCLE_CHOLQR = 0, LSBA_MUSCLE_COLUMN = 1 };

/* Counters and outcome of the last lsba_solve. */
typedef struct {
  int32_t status;
  int32_t cycles;          /* restart cycles run                                 */
  int32_t steps;           /* completed Arnoldi relations over all cycles        */
  int32_t a_calls;         /* applications of A (SpMM launches that did work)    */
  int32_t syncs;           /* sync points: block inner products + IntraOrtho     */
  int32_t v_apps;          /* applications of the basis (paper's counting)       */
  int32_t flags;           /* Cholesky NaN-flags raised                          */
  int32_t m_final;         /* maximum basis size in force at the end             */
  double relres_est;       /* last residual estimate ||[M;-H] c C||_F / ||B||_F  */
  double relres_true;      /* ||B - A X||_F / ||B||_F (NaN if not computed)       */
  double solve_ms;         /* wall time of lsba_solve                            */
  int32_t precision;       /* precision the solve ran in (LSBA_PREC_*)           */
  int32_t ir_outer;        /* FP32_IR: refinement steps (inner solves) taken     */
  int32_t tensor_cores;    /* 1: the Gram and update passes of the Arnoldi steps
                              ran on the tensor-core digit kernels               */
} lsba_stats;

/* Host-side copies kept by the handle when record_history = 1; valid until the
 * next lsba_solve or lsba_destroy.  Matrices are column-major. */
typedef struct {
  int32_t n_est;                 /* entries in est / est_cycle / est_j             */
  const double* est;             /* residual estimate after each relation          */
  const int32_t* est_cycle;      /* its cycle (1-based)                            */
  const int32_t* est_j;          /* its relation index j                           */
  int32_t n_cycles;
  const int32_t* cycle_m;        /* relations completed per cycle                  */
  const int32_t* cycle_flag;     /* relation that flagged per cycle (0 none)       */
  const int32_t* cycle_mcur;     /* maximum basis size in force per cycle          */
  int32_t first_j;               /* relations completed in the first cycle         */
  const double* first_H;         /* (first_j+1)s x first_j*s, ld = (first_j+1)s    */
  const double* first_beta;      /* s x s, the CholQR factor of B                  */
  int32_t n_grams;               /* skeleton inner products recorded, first cycle  */
  const int32_t* gram_rows;      /* rows of each (row-major data, concatenated)    */
  const int32_t* gram_cols;
  const double* gram_data;
} lsba_history;

/* Fill *opt with the defaults. */
void lsba_default_options(lsba_options* opt);

/* Create a solver handle on `device`, ordered on `cuda_stream` (a cudaStream_t).
 * NULL: the handle creates a blocking stream of its own, which the legacy
 * default stream orders implicitly against its own work (the same ordering as
 * launching on the legacy default stream, which cannot be captured into a
 * graph).  opt may be NULL (defaults).  The handle owns its workspace,
 * allocated on first use and grown on demand. */
int lsba_create(lsba_handle* out, int device, void* cuda_stream, const lsba_options* opt);

/* Replace the handle's options. */
int lsba_set_options(lsba_handle h, const lsba_options* opt);

/* Solve A X = B with restarted block Arnoldi of maximum basis size m (m >= 1,
 * (m+1)*s <= 2048) to relative residual tol: ||B - A X||_F / ||B||_F <= tol
 * (by the estimate of Eq. (9), confirmed on the true residual when
 * verify_true_residual is set).  X_0 = 0.
 *   A:   CSR on the device (see lsba_csr)
 *   d_B: n x s input, d_X: n x s output (the caller's device buffers)
 * Returns LSBA_OK, LSBA_NOT_CONVERGED (X = last iterate), LSBA_BREAKDOWN, or an
 * error code. */
int lsba_solve(lsba_handle h, const lsba_csr* A, const double* d_B, double* d_X,
               int s, int m, double tol, lsba_skeleton skel);

/* Same solve with HOST buffers for the matrix and the blocks: the handle copies
 * A and B to the device, solves, and copies X back (timed end to end). */
int lsba_solve_host(lsba_handle h, int64_t n, int64_t nnz, const int32_t* h_rowptr,
                    const int32_t* h_colidx, const double* h_vals, const double* h_B,
                    double* h_X, int s, int m, double tol, lsba_skeleton skel);

int lsba_get_stats(lsba_handle h, lsba_stats* out);

/* Return the handle's device workspace to the device memory pool (stream-ordered
 * on the handle's stream; no device-wide synchronisation).  The next solve
 * allocates again.  All workspace allocations of the library are stream-ordered
 * (cudaMallocAsync / cudaFreeAsync), so solves on different handles and
 * streams can run, grow and release concurrently. */
int lsba_release_workspace(lsba_handle h);

/* Upper bound of the device memory (bytes) lsba_solve with n x s blocks, nnz
 * nonzeros and basis size m allocates on the current device, for admission
 * control (lsba_solve_host adds its own copies of A, B and X); -1 on invalid
 * sizes.  Host computation only; with no device visible it assumes 256 SMs,
 * which bounds the Gram partial sums of any current part.  The restart
 * history of lsba_get_history keeps at most 4096 cycles. */
int64_t lsba_workspace_bytes(int64_t n, int64_t nnz, int s, int m);

/* Kernel classes of lsba_get_profile. */
enum { LSBA_K_SPMM = 0, LSBA_K_GRAM = 1, LSBA_K_UPDATE = 2, LSBA_K_SMALL = 3, LSBA_K_NCLASS = 4 };

/* Device time (ms, from CUDA events recorded around each launch on the
 * handle's stream) and launch counts per kernel class, accumulated over the
 * solves since the last lsba_reset_profile, when options.profile = 1.
 * ms and launches are caller arrays of nclass entries (nclass <= LSBA_K_NCLASS). */
int lsba_get_profile(lsba_handle h, double* ms, int64_t* launches, int nclass);
int lsba_reset_profile(lsba_handle h);
int lsba_get_history(lsba_handle h, lsba_history* out);
const char* lsba_status_string(int status);
int lsba_destroy(lsba_handle h);

/* ---- kernel-level entry points (one hot-path step each; used for parity and
 * roofline measurement).  All are blocking on the handle's stream. ---------- */

/* W = A V  (the paper's matvec on a block vector, Sec. 2.1).  V, W: n x s. */
int lsba_spmm(lsba_handle h, const lsba_csr* A, const double* d_V, double* d_W, int s);

/* Block inner product G = [L_1 .. L_a]^T [R_1 .. R_b] (Table 1; the one-pass
 * sync point of Alg. 3 line 4, Alg. 6 line 10, Alg. 7 line 10).
 *   d_L: a blocks of n x s, contiguous ([a][n][s]); d_R: b blocks likewise.
 *   d_G: (a*s) x (b*s) output, row-major.  1 <= a <= 2048/s, 1 <= b <= 2.
 * Summation order is fixed: the result is bitwise reproducible run to run. */
int lsba_gram(lsba_handle h, const double* d_L, int a, const double* d_R, int b,
              int64_t n, int s, double* d_G);

/* Autotuner of the double-float lagged skeletons (BCGSI+LS, BMGS-CWY/ICWY) for
 * any block size s (Sec. 2.1 treats the inner product and the basis update as
 * separately tunable functions).  For every iteration k = 2..m+1 of a cycle it
 * times, on the handle's stream with CUDA events (one warm-up and three runs
 * each, on pseudo-random n x s operands whose digits are all busy, and their
 * stored digit planes where a kernel reads them), the candidate shapes of the
 * iteration's two passes and keeps the fastest:
 *   Gram [V_1..V_{k-1}, U]^T [U, W] (Alg. 7 line 10): the FP32-pipe kernel
 *     with 1..4 CTAs per SM and its default or half its pipeline chunk rows
 *     (shapes whose shared memory cannot stay resident at that CTA count are
 *     skipped), the split-digit tensor-core kernel where its shape allows, and
 *     at s = 8 the stored-digit tensor-core kernel (tensor-core candidates only
 *     when options.tensor_cores != 0);
 *   update (Alg. 7 lines 16-17): at s = 8 with tensor cores the stored-digit
 *     tensor-core update with two or three CTAs per SM, else the FP32-pipe
 *     update with 1, 2, 4 or 8 CTAs per SM.
 * Later solves on this handle with the same n and s run the tuned shape at each
 * k (otherwise fixed rules: the stored-digit Gram from k = 5, the FP32-pipe
 * kernels' default grids).  Kernels round differently (all to 48-bit
 * accuracy), so tuned and untuned solves agree to rounding, not bit for bit;
 * the shapes of one kernel give the same bits.  The workspace is (re)allocated
 * for (n, s, m); the basis contents are overwritten.
 * gram_choice[k] (k < cap): 0 FP32-pipe Gram, 1 split-digit tensor-core Gram,
 * 2 stored-digit tensor-core Gram, -1 no choice; update_ctas[k]: CTAs per SM of
 * the chosen update, 0 no choice.  Host arrays of cap entries (may be NULL when
 * cap = 0).  Returns LSBA_OK, LSBA_INVALID_ARG (n < 1, s outside 1..32, m < 1
 * or (m + 1) s too large), LSBA_OUT_OF_MEMORY, LSBA_DEVICE_TIMEOUT or
 * LSBA_CUDA_ERROR. */
int lsba_autotune(lsba_handle h, int64_t n, int s, int m, int8_t* gram_choice,
                  int8_t* update_ctas, int cap);

/* One tuned iteration of the last lsba_autotune on this handle. */
typedef struct {
  int32_t k;                    /* iteration (its Gram reads k + 1 blocks) */
  int32_t gram_kernel;          /* 0 FP32 pipe, 1 split-digit tensor cores, 2 stored-digit tensor cores */
  int32_t gram_ctas_per_sm;     /* FP32-pipe Gram: CTAs per SM (else 0) */
  int32_t gram_rows;            /* FP32-pipe Gram: cap on the rows of a pipeline chunk (0: default) */
  int32_t update_kernel;        /* 0 FP32-pipe update, 1 stored-digit tensor-core update */
  int32_t update_ctas_per_sm;   /* CTAs per SM of that update */
  float gram_us;                /* measured time of the chosen Gram shape, microseconds a launch */
  float update_us;              /* measured time of the chosen update shape, microseconds a launch */
  float gram_default_us;        /* the untuned rule's Gram, microseconds (0: not measured) */
  float update_default_us;      /* the untuned rule's update, microseconds */
} lsba_tune_entry;

/* The table of the last lsba_autotune (iterations in increasing k): *count is
 * the number of entries, of which the first min(cap, *count) are written to
 * out (host array).  LSBA_OK, or LSBA_INVALID_ARG for a NULL handle, count,
 * or out with cap > 0. */
int lsba_autotune_table(lsba_handle h, lsba_tune_entry* out, int cap, int* count);

/* The same G as lsba_gram, computed by the double-float Gram kernels of the
 * solver (the block inner product of every skeleton, Sec. 2): L and R are
 * converted to hi + lo FP32 pairs on the device, G is returned in FP64.
 * tensor_cores = 1 selects the tensor-core digit kernel wherever its shape
 * allows (s % 4 == 0, b s <= 16, (a + b) s <= 256), 0 the FP32-pipe kernel,
 * 3 the tensor-core kernel on stored digit planes that the solver uses for a
 * lagged skeleton's basis (s = 8, b = 2, 2 <= a, a s <= 168): L_1..L_{a-1}
 * are split into digit planes first and R_1 stands for L_a, so the result is
 * [L_1..L_{a-1}, R_1]^T [R_1, R_2].  b <= 2.
 * Temporary copies are allocated stream-ordered on the handle's stream and
 * released before return.  LSBA_DEVICE_TIMEOUT if a kernel's bounded wait
 * gave up.  With options.profile = 1 the Gram kernels' device time (without
 * the conversions) is added to the LSBA_K_GRAM class of lsba_get_profile. */
int lsba_gram_df(lsba_handle h, const double* d_L, int a, const double* d_R, int b, int64_t n,
                 int s, double* d_G, int tensor_cores);

/* Block combination (the basis update of Alg. 3 line 6 / Alg. 7 lines 16-17):
 *   out[r,:] = ( sum_i in_i[r,:] * C_i ) * T^{-1}
 *   d_in: nin blocks n x s contiguous; d_C: nin*s x s row-major (block i of rows
 *   is C_i); d_T: s x s upper-triangular (row-major) or NULL for no solve. */
int lsba_combine(lsba_handle h, const double* d_in, int nin, int64_t n, int s,
                 const double* d_C, const double* d_T, double* d_out);

/* FP64 on the tensor cores (exact digit products; the Gram and update passes
 * the solver runs for BCGSI+LS and BMGS-CWY/ICWY at s = 8 in FP64).
 * Every FP64 value is split, relative to the maximum of its (128-row tile,
 * column) group, into seven 8-bit digits carrying 53 bits (F = trunc(x
 * 2^(54 - E)) for max |x| < 2^E); the fp16 tensor cores sum the digit products
 * by level exactly in FP32 over windows of at most 128 products, and each
 * window's levels 0..7 are combined in 64-bit integers and added into FP64
 * accumulators.  Error per product term about 2^-53 (max|x| |y| + |x| max|y|).
 *
 * lsba_gram_fp64tc: G = [L_1..L_a]^T [R_1..R_b], the Gram of lsba_gram (same
 *   layouts), s = 8, a*s <= 256, b <= 2, a + b <= 24; deterministic (fixed
 *   reduction order).
 * lsba_combine_fp64tc: out1 = ([in_1..in_nin] C1) T^{-1} (d_T: s x s upper,
 *   row-major, or NULL) and, if d_out2, out2 = [in_1..in_nin] C2; C1, C2 are
 *   nin*s x s row-major (block i of rows multiplies in_i); s = 8, nin <= 24.
 * Both return LSBA_OK, LSBA_INVALID_ARG (shape outside these limits),
 * LSBA_OUT_OF_MEMORY, LSBA_CUDA_ERROR or LSBA_DEVICE_TIMEOUT (a bounded wait
 * inside the kernel gave up). */
int lsba_gram_fp64tc(lsba_handle h, const double* d_L, int a, const double* d_R, int b,
                     int64_t n, int s, double* d_G);
int lsba_combine_fp64tc(lsba_handle h, const double* d_in, int nin, int64_t n, int s,
                        const double* d_C1, const double* d_T, const double* d_C2,
                        double* d_out1, double* d_out2);

/* ---- allocation-free variant ------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory: serving loops that must not pay for an
 * allocation or the synchronisation cudaFree implies, and hosts that fix the
 * device memory footprint at start-up (a budget shared with other processes,
 * or an allocator that owns the device's memory).
 *
 * lsba_gram_noalloc computes the same G = [L_1..L_a]^T [R_1..R_b] as lsba_gram
 * (same arguments and layouts) without a handle and without allocating: no
 * cudaMalloc, cudaFree or allocating library routine is called.  Its partial
 * sums live in a fixed array in the library's device memory of
 * LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES doubles (512 KiB), which every GPU that loads
 * the library holds until the process exits.
 *   - Limit: (a*s)*(b*s) <= LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES, otherwise
 *     LSBA_INVALID_ARG is returned and nothing is launched.  The partial sums
 *     take one row of (a*s)*(b*s) doubles per row partition (one CTA each), so
 *     at most LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES / ((a*s)*(b*s)) partitions fit:
 *     where lsba_gram would use more, this call uses fewer CTAs and runs at
 *     lower bandwidth than lsba_gram (e.g. a*s = 168, b*s = 16: 24 CTAs).
 *   - Errors: if a CUDA error is already pending when the call starts (left
 *     by earlier work of the caller), it returns LSBA_CUDA_ERROR without
 *     launching and leaves that error pending; an error of its own launch is
 *     cleared and reported as LSBA_CUDA_ERROR.
 *   - Device: the current CUDA device.  The first call on a device looks up the
 *     array's device address (cudaGetSymbolAddress) and caches it; make that
 *     first call before any stream capture.
 *   - Ordering: enqueued on cuda_stream (NULL = legacy default stream); the
 *     call returns without waiting.  Every call shares the one array and
 *     overwrites all of it that it reads, so no clearing is needed, but calls
 *     whose kernels overlap on the GPU (different streams, or different host
 *     threads) race on it and must be serialised by the caller.
 * Returns LSBA_OK, LSBA_INVALID_ARG or LSBA_CUDA_ERROR. */
#define LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES (1 << 16)
int lsba_gram_noalloc(const double* d_L, int a, const double* d_R, int b, int64_t n, int s,
                      double* d_G, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LSBA_H */
