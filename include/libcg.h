/*
 * libcg — sparse (preconditioned) conjugate gradient on one GB300 GPU (sm_103a).
 *
 * C ABI of the CG hot path of "A Preliminary Study on Simultaneous
 * Coscheduling for Discrete GPU vs. Fused GPU" (ICPP Workshops '26), run
 * entirely on the GPU (the paper's GPU-only split, g = 1).  The paper's
 * problem statement (Sec. 3): solve A x = b for a sparse A that stays fixed
 * during the solve, A held in CSR form (Sec. 3.2) with fp64 values, vectors
 * and reductions (Sec. 3.1), each iteration = fused SpMV + p.q, fused x/r
 * update + r.r, p update (Alg. 1, Sec. 3.3).
 *
 * Conventions for every call:
 *  - Pointers named in the comments as "device" must point to memory of the
 *    current CUDA device; "host" pointers to ordinary or pinned host memory.
 *  - Matrix arrays are BORROWED: the caller keeps rowptr/colind/vals alive and
 *    unchanged until cg_destroy.  Every other buffer the library needs is
 *    allocated (cudaMalloc) by cg_create and freed by cg_destroy.
 *  - Indices are int32 (0-based), values fp64; vectors are fp64 with 16-byte
 *    aligned start addresses (any torch.empty/zeros tensor qualifies).
 *  - Work is ordered on the handle's stream (cg_set_stream; default: the
 *    legacy default stream).  cg_solve blocks until its result word is back
 *    on the host; cg_spmv does not block.
 *  - Every call returns a cg_status.  CG_NOT_CONVERGED is not an error: the
 *    outputs are valid.  Negative values are errors; cg_last_error() gives a
 *    one-line reason.  A handle is not thread-safe.
 */
#ifndef LIBCG_H
#define LIBCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cg_handle cg_handle;

typedef enum {
  CG_OK = 0,
  CG_NOT_CONVERGED = 1,   /* maxit reached (or restarts exhausted); x is the last iterate */
  CG_ERR_INVALID = -1,    /* bad argument, malformed CSR, missing/non-positive diagonal */
  CG_ERR_BREAKDOWN = -2,  /* p.q <= 0: A is not SPD on the Krylov space */
  CG_ERR_NUMERIC = -3,    /* NaN or Inf in a reduction */
  CG_ERR_TIMEOUT = -4,    /* a bounded wait gave up: a grid barrier of the persistent kernel or an
                             exchange of partial sums in the cluster form */
  CG_ERR_CUDA = -5,       /* a CUDA runtime call failed */
  CG_ERR_OOM = -6         /* device or pinned-host allocation failed */
} cg_status;

typedef enum {
  CG_PRECOND_NONE = 0,    /* plain CG, Alg. 1 */
  CG_PRECOND_JACOBI = 1,  /* z = D^-1 r, D = diag(A) (not in the paper) */
  CG_PRECOND_FSAI = 2     /* z = G^T G r with the handle's FSAI factor G (cg_fsai_classic,
                             cg_fsai_load, cg_fsai_set_factor; not in the paper); without
                             a factor the solve falls back to Jacobi (precond_used says so) */
} cg_precond;

typedef enum {
  CG_PREC_FP64 = 0,       /* every value, vector and reduction in fp64 (Sec. 3.1) */
  CG_PREC_FP32_IR = 1,    /* fp32 inner PCG, fp64 outer iterative refinement (not in the paper) */
  CG_PREC_FP32_RU = 2     /* fp32 PCG with fp64 reliable updates: as CG_PREC_FP32_IR, but the
                             search direction survives each fp64 update (p = z' + (r'.z'/rho) p)
                             instead of restarting, so the iteration count stays close to fp64
                             PCG's (not in the paper); persistent loop form only */
} cg_precision;

typedef enum {
  CG_OPT_MAX_RESTARTS = 0,        /* residual-replacement restarts after a false convergence (default 3) */
  CG_OPT_BARRIER_TIMEOUT_MS = 1,  /* limit of every bounded wait in ms (default 2000) */
  CG_OPT_GRID_CTAS = 2,           /* persistent-kernel CTAs; 0 = choose automatically (default) */
  CG_OPT_IR_TOL_INNER = 3,        /* inner relative tolerance of fp32 refinement (default 1e-4), or the
                                     residual reduction that triggers a reliable update (default 0.1) */
  CG_OPT_IR_MAX_OUTER = 4,        /* refinement steps / reliable updates cap (default 30) */
  CG_OPT_DEBUG_SKIP_ARRIVAL = 5,  /* fault injection: CTA 0 skips arrival at grid barrier #value
                                     (cluster form: does not push exchange #value; 1-based; 0 = off),
                                     so every wait runs into its limit */
  CG_OPT_PHASE_TIMERS = 6,        /* 1: record CTA 0's time per loop phase in cg_solve_info */
  CG_OPT_LOOP_MODE = 7            /* loop form: 0 auto (fp64 Jacobi / plain CG: cluster form up to
                                     16384 rows unless CG_OPT_GRID_CTAS, CG_OPT_DEBUG_SKIP_ARRIVAL
                                     or CG_OPT_PHASE_TIMERS is set, graph from 2^18 rows; fp32
                                     FSAI refinement: graph from 2^21 rows; else persistent),
                                     1 one persistent cooperative launch, 2 CUDA graph with a
                                     device-side WHILE node (nested WHILE nodes for fp32
                                     refinement), 3 graphs of 8 unrolled iterations relaunched by
                                     the host until done (fp64 Jacobi / plain CG and the fp32
                                     FSAI refinement; elsewhere as 2), 4 one thread-block cluster
                                     of up to 16 CTAs holding the whole system in shared memory
                                     (fp64 Jacobi / plain CG, at most 32768 rows; the debug and
                                     timer options have no effect there).  The Jacobi
                                     reliable-update solve and the fp64 FSAI solve always take
                                     form 1. */
} cg_option;

/* Statistics of the most recent cg_solve on a handle. */
typedef struct {
  int32_t status;         /* cg_status of the solve */
  int32_t iters;          /* SpMVs in the CG loop (fp64) / total inner iterations (fp32 IR) */
  int32_t restarts;       /* residual replacements (fp64) / refinement steps (fp32 IR) */
  int32_t grid_ctas;      /* CTAs of the persistent launch */
  double relres_true;     /* ||b - A x||_2 / ||b||_2 recomputed in fp64 from the final x */
  double relres_rec;      /* the recursive residual's relative norm at exit */
  double kernel_ms;       /* device time of the persistent launch (CUDA events) */
  int64_t bytes_moved;    /* modelled HBM bytes of the loop: iters x (12 nnz + 4(n+1) + 104 n)
                             (Jacobi; 88 n without; fp32 refinement 8 nnz + 4(n+1) + 52/44 n) */
  int64_t kernel_bytes_per_iter; /* bytes one iteration of this library's loop must move:
                             its off-diagonal slices (fp64: 8 B/entry in the diagonal layout,
                             12 B with a column array; fp32: 4 / 8 B) plus 88 n (Jacobi) /
                             80 n bytes of vectors (fp64; half that in fp32) */
  double phase_ms[6];     /* with CG_OPT_PHASE_TIMERS: CTA 0 time in the SpMV, r-update and
                             x/p-update phases, each followed by its grid-barrier wait */
  int32_t loop_form;      /* CG_OPT_LOOP_MODE form that ran: 1 persistent, 2 graph WHILE, 3 unrolled,
                             4 cluster */
  int32_t kernel_launches;/* kernels of this library launched by the solve */
  int32_t precond_used;   /* cg_precond that ran (CG_PRECOND_FSAI without a factor runs Jacobi) */
} cg_solve_info;

/*
 * Create a solver for the n x n CSR matrix (rowptr[n+1], colind[nnz],
 * vals[nnz], all DEVICE pointers, nnz = rowptr[n]).  The CSR is validated
 * (rowptr[0] = 0, non-decreasing, every colind in [0, n)); the diagonal is
 * extracted for Jacobi (a row whose diagonal is absent or <= 0 only disables
 * Jacobi).  The rows are cut into row blocks for the SpMV schedule.  On
 * success *out owns all workspace; on failure *out = NULL and the status says
 * why (message via cg_last_error(NULL)).  n = 0 is allowed.
 */
cg_status cg_create(int64_t n, const int32_t* rowptr, const int32_t* colind,
                    const double* vals, cg_handle** out);

/* Order all later work of h on `cuda_stream` (a cudaStream_t; NULL = legacy default). */
cg_status cg_set_stream(cg_handle* h, void* cuda_stream);

/* Set a tuning/debug option (cg_option); returns CG_ERR_INVALID for unknown options or values. */
cg_status cg_set_option(cg_handle* h, int32_t option, double value);

/* y = A x (Sec. 3.1 SpMV), x and y DEVICE fp64 vectors of length n; y must not alias x. */
cg_status cg_spmv(cg_handle* h, const double* x, double* y);

/*
 * Solve A x = b (Alg. 1).  b: DEVICE rhs; x: DEVICE, in = initial guess x0,
 * out = solution.  Stops when ||r||_2 <= tol ||b||_2 on the recursive
 * residual (tested before each SpMV, so iters counts SpMVs), then recomputes
 * the true residual in fp64; if that misses tol, restarts from x (residual
 * replacement) up to CG_OPT_MAX_RESTARTS times.  b = 0 gives x = 0, iters 0,
 * relres 0.  The loop runs either as one persistent cooperative launch or
 * as one launch of a captured CUDA graph whose WHILE node the kernels
 * themselves continue or end (CG_OPT_LOOP_MODE picks the form; auto takes
 * the graph for large fp64 systems); either way there is no host round trip
 * per iteration.  iters_out / relres_out (host, may be NULL)
 * receive the iteration count and the fp64 true relative residual.
 * Returns CG_OK, CG_NOT_CONVERGED or an error (x then holds the last iterate).
 */
cg_status cg_solve(cg_handle* h, const double* b, double* x, double tol, int32_t maxit,
                   int32_t precond, int32_t precision, int32_t* iters_out, double* relres_out);

/*
 * cg_solve with HOST buffers: b_host and x_host (x0 in, solution out) are
 * copied to the device and back inside the call (pinned memory makes the
 * copies asynchronous and fastest).  Same results and statuses as cg_solve.
 */
cg_status cg_solve_host(cg_handle* h, const double* b_host, double* x_host, double tol,
                        int32_t maxit, int32_t precond, int32_t precision, int32_t* iters_out,
                        double* relres_out);

/*
 * Build everything cg_solve(precond, precision) needs on this handle (the
 * loop matrix in its sliced layout, scaled by D^-1/2 for Jacobi, the fp32
 * copy for the refinement precisions, the work vectors), so that the first
 * solve does no setup work.  Optional: cg_solve builds whatever is missing.
 * Synchronous.  Errors as cg_solve's argument checks; CG_ERR_OOM when an
 * allocation fails.
 */
cg_status cg_prepare(cg_handle* h, int32_t precond, int32_t precision);

/*
 * The solve loop's own SpMV kernel on its own: q = A^ p with A^ = D^-1/2 A
 * D^-1/2 for CG_PRECOND_JACOBI and A otherwise (Sec. 3.1 SpMV on the loop
 * matrix of Alg. 1), fused with the p.q reduction exactly as in each loop
 * iteration of the graph form (the reduction's result stays on the device).
 * p and q are DEVICE vectors of n doubles (CG_PREC_FP64) or n floats (the
 * fp32 precisions), 16-byte aligned, not aliased.  The kernel is launched
 * reps >= 1 times back to back on the handle's stream (after one tiny state
 * kernel); the call does not block.  *bytes_out (host, may be NULL) gets the
 * bytes one launch must move: the loop matrix entries (values, plus int32
 * columns when the matrix is not in the diagonal layout), p read once, q
 * written (and the stored diagonal without Jacobi).
 */
cg_status cg_loop_spmv(cg_handle* h, int32_t precond, int32_t precision, const void* p, void* q,
                       int32_t reps, int64_t* bytes_out);

/* Statistics of the last solve on h (host struct). */
cg_status cg_get_solve_info(const cg_handle* h, cg_solve_info* out);

/* Matrix and schedule facts: n, nnz, row blocks, long rows, CTAs of the persistent kernel. */
cg_status cg_get_matrix_info(const cg_handle* h, int64_t* n, int64_t* nnz, int64_t* row_blocks,
                             int64_t* long_rows, int32_t* grid_ctas);

/* Free every buffer owned by h (not the borrowed CSR).  NULL is a no-op. */
void cg_destroy(cg_handle* h);

/* Last error message of h, or of the calling thread's last failed cg_create when h is NULL. */
const char* cg_last_error(const cg_handle* h);

/* Static name of a status code. */
const char* cg_status_string(int32_t status);

/* Most systems in one batch handle. */
#define CG_BATCH_MAX_SYSTEMS 4096

/*
 * Create a solver for nsys independent systems (1 <= nsys <=
 * CG_BATCH_MAX_SYSTEMS) of uneven size, all solved by one launch.  n[s]
 * (host array, each >= 1) is the order of system s; rowptr[s], colind[s] and
 * vals[s] (host arrays of DEVICE pointers) its CSR, validated as in
 * cg_create and borrowed until cg_destroy.  The handle concatenates the
 * systems into one block-diagonal matrix in 256-row tiles (so it holds a
 * second copy of all matrices: a system whose off-diagonal entries lie on at
 * most 8 offsets by diagonal, the others as sliced ELL) and serves
 * cg_solve_batch,
 * cg_batch_get_system, cg_batch_get_tuning, cg_set_stream, cg_set_option,
 * cg_get_solve_info, cg_last_error and cg_destroy; the single-system calls
 * return CG_ERR_INVALID on it.  On failure *out = NULL and
 * cg_last_error(NULL) names the system at fault.
 */
cg_status cg_batch_create(int32_t nsys, const int64_t* n, const int32_t* const* rowptr,
                          const int32_t* const* colind, const double* const* vals,
                          cg_handle** out);

/*
 * Solve every system of a batch handle, each exactly as cg_solve would alone
 * (Alg. 1 with the same stopping rule, fp64 true-residual test and restarts).
 * precision: CG_PREC_FP64; CG_PREC_FP32_IR (fp32 inner PCG on the fp32 loop
 * matrix, fp64 residual, x += d and test per refinement step, inner tolerance
 * CG_OPT_IR_TOL_INNER, default 1e-4); CG_PREC_FP32_RU (the same with the
 * search direction carried over each fp64 update, default inner drop 0.1);
 * CG_OPT_IR_MAX_OUTER caps the refinement steps of each system.  b[s] and
 * x[s] (host arrays of DEVICE pointers, length n[s]) are system s's rhs and
 * initial guess / solution.  One persistent cooperative kernel, captured with
 * its gather and scatter kernels in a CUDA graph (CG_OPT_LOOP_MODE 1: direct
 * launch), iterates all systems; a converged system drops out of the tile
 * schedule.  The kernel variant (registers budgeted for 3, 4 or 5 resident
 * CTAs per SM) and grid size come from an autotuner that times short trial
 * solves of these systems at the first solve of each (preconditioner,
 * precision kind) (x is not touched by the trials; the choice is kept in the
 * handle); CG_OPT_GRID_CTAS > 0 forces the grid instead.  iters[s] and
 * relres[s] (host, may be NULL) receive each system's iterations (fp64 PCG
 * steps, or inner fp32 steps in all) and fp64 true relative residual.
 * Returns the most severe error of any system, else CG_NOT_CONVERGED if any
 * system missed tol, else CG_OK; per-system results via cg_batch_get_system
 * (restarts = residual replacements in fp64, refinement steps / updates in
 * fp32).  cg_get_solve_info reports the largest iteration count and residual,
 * the grid, the device time and the modelled bytes summed over systems.
 */
cg_status cg_solve_batch(cg_handle* h, const double* const* b, double* const* x, double tol,
                         int32_t maxit, int32_t precond, int32_t precision, int32_t* iters,
                         double* relres);

/* Result of system s (0 <= s < nsys) of the last cg_solve_batch: status, iterations,
 * restarts and fp64 true relative residual (each pointer may be NULL). */
cg_status cg_batch_get_system(const cg_handle* h, int32_t s, int32_t* status, int32_t* iters,
                              int32_t* restarts, double* relres);

/* The autotuner's record for a preconditioner and precision (both fp32
 * precisions share one record): *count candidates (kernel variant = resident
 * CTAs per SM its registers are budgeted for, grid size) with their trial
 * times in ms (arrays of at least 8 entries, may be NULL), and the index of
 * the chosen candidate (-1 before the first autotuned solve). */
cg_status cg_batch_get_tuning(const cg_handle* h, int32_t precond, int32_t precision, int32_t* count,
                              int32_t* grids, int32_t* ctas_per_sm, float* ms, int32_t* chosen);

/*
 * FSAI preconditioner M^-1 = G^T G (Kolotilina & Yeremin 1993; not in the
 * paper).  G is lower triangular with the pattern of tril(A); the CSR of A
 * must have strictly increasing columns in every row, a positive diagonal,
 * at most 16 entries per row of tril(A) and at most 32 per column.  The
 * factor belongs to the handle and is used by cg_solve(precond =
 * CG_PRECOND_FSAI) in both precisions (fp32 refinement: G rounded to fp32);
 * each iteration applies it as t = G r, z = G^T t (three grid barriers per
 * iteration, as with Jacobi).  The pattern of G and G^T is built once per
 * handle, on the device when the CSR's structure is symmetric (else on the
 * host); the factor calls synchronise the handle's stream.
 */

/* Classic FSAI: per row i, solve A[P_i,P_i] y = e_i on the row's pattern P_i
 * (small dense Cholesky on the GPU) and set row i of G to y / sqrt(y_i).
 * CG_ERR_INVALID if the matrix does not qualify or a local matrix is not SPD. */
cg_status cg_fsai_classic(cg_handle* h);

/* Use the caller's factor: g_tril (DEVICE, fp64) holds G's values in the
 * order of the entries of tril(A) in A's CSR (row by row, columns
 * ascending).  Every diagonal value must be positive and finite. */
cg_status cg_fsai_set_factor(cg_handle* h, const double* g_tril);

/* Copy the current factor (tril order) into g_tril (DEVICE, may be NULL);
 * *ntril = nonzeros of tril(A), *kind = 0 none, 1 classic, 2 learned, 3 set. */
cg_status cg_fsai_get_factor(cg_handle* h, double* g_tril, int64_t* ntril, int32_t* kind);

/*
 * Learned FSAI factor (not in the paper): an MLP with CG_MLP_INPUTS inputs,
 * two hidden ReLU layers of CG_MLP_HIDDEN units and one output maps local
 * features of every entry (i, j) of tril(A) to G_ij.  Features (A_ii = d_i,
 * s(i,k) = A_ik / sqrt(d_i d_k)): [0:8] one-hot slot of j - i among the
 * non-positive column offsets of A; [8] s(i,j); [9] log(d_j / d_i); [10:19]
 * s(i, i + o_m) and [19:28] s(j, j + o_m) over the sorted distinct column
 * offsets o_m of A (the matrix may have at most 9); [28] 1; [29:32] 0.
 * Output o: G_ij = o / sqrt(d_j) for j < i and G_ii = softplus(o + c0) /
 * sqrt(d_i) with softplus(c0) = 1, so a zero output layer is Jacobi.
 * Parameters, in this order (row-major, a row per output unit):
 *   W1[64][32], b1[64], W2[64][64], b2[64], W3[64], b3  (CG_MLP_PARAMS values).
 * Layers 1 and 2 run on the tensor cores with bf16 inputs and fp32 sums.
 */
#define CG_MLP_INPUTS 32
#define CG_MLP_HIDDEN 64
#define CG_MLP_PARAMS 6337

/* Compute the handle's factor with the MLP (inference).  weights_bf16: HOST
 * array of CG_MLP_PARAMS bfloat16 values (bytes = 2 * CG_MLP_PARAMS). */
cg_status cg_fsai_load(cg_handle* h, const void* weights_bf16, int64_t bytes);

/* cg_fsai_load from fp32 weights: weights is a HOST array of count =
 * CG_MLP_PARAMS floats, rounded to bf16 (nearest, ties to even) by the
 * library.  CG_ERR_INVALID for a wrong count, a NaN or infinite weight, or a
 * finite weight that rounds beyond the largest bf16 value. */
cg_status cg_fsai_load_f32(cg_handle* h, const float* weights, int64_t count);

/*
 * Training loss of the MLP on the handle's matrix and its gradient.
 * params: DEVICE fp32[CG_MLP_PARAMS] (rounded to bf16 for the forward pass);
 * grad: DEVICE fp32[CG_MLP_PARAMS], overwritten with dLoss/dparams; resid:
 * DEVICE fp64[nresid][n] residual vectors r_k (may be NULL when nresid = 0).
 *   Loss = log((1/n) sum_i g_i^T A g_i) - (2/n) sum_i log G_ii      (Kaporin)
 *        + lambda (1/K) sum_k ||A G^T G r_k - r_k||^2 / ||r_k||^2.
 * *loss_out (host) receives the loss.  Reductions run in a fixed order: the
 * same inputs give the same bits.  Does not change the handle's factor.
 */
cg_status cg_fsai_loss_grad(cg_handle* h, const float* params, float* grad, const double* resid,
                            int32_t nresid, double lambda, double* loss_out);

/* One Adam step (Kingma & Ba) on DEVICE fp32 arrays of count values:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps); step >= 1.
 * Enqueued on cuda_stream (a cudaStream_t, NULL = legacy default stream). */
cg_status cg_adam_step(float* params, const float* grad, float* m, float* v, int64_t count, float lr,
                       float beta1, float beta2, float eps, int32_t step, void* cuda_stream);

/* Largest n that cg_solve_noalloc accepts: its scratch is four device vectors
 * of this many doubles plus a result block (2 MiB per GPU). */
#define CG_NOALLOC_MAX_ROWS 65536

/*
 * Allocation-free (Jacobi-)CG for small systems.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory: a
 * plugin or operator inside a framework that owns all device memory through
 * its own pool, code that may not hold device allocations of its own, or a
 * latency-critical loop where a cudaMalloc could synchronise the device.
 *
 * It needs no handle and calls no cudaMalloc/cudaFree: the scratch vectors
 * live in one file-scope __device__ array that every GPU loading this library
 * keeps until the process exits.  n <= CG_NOALLOC_MAX_ROWS; rowptr[n+1],
 * colind[nnz], vals[nnz], b[n] and x[n] are DEVICE pointers (x: x0 in,
 * solution out); cuda_stream is a cudaStream_t (NULL = legacy default);
 * iters_out / relres_out are host pointers and may be NULL.  The solve follows
 * cg_solve's rules (relative test before each SpMV, fp64 true residual, up to
 * 3 residual-replacement restarts) but runs in a single CTA, so it suits small
 * systems only.  It blocks until the result is on the host.
 *
 * Errors: CG_ERR_INVALID when n exceeds CG_NOALLOC_MAX_ROWS, a size or
 * pointer is bad, the CSR is malformed (checked on the device: rowptr[0] = 0,
 * rowptr[n] = nnz, non-decreasing, colind in [0, n)) or Jacobi meets a row
 * without a positive diagonal; CG_ERR_CUDA when a CUDA call fails; otherwise
 * the statuses of cg_solve.
 *
 * All calls on a device share the scratch array, which keeps the last call's
 * contents (the kernel initialises what it reads): calls that may overlap on
 * the GPU (other streams or host threads) race and must be serialised by the
 * caller.  The first call on each device looks up the array's device address
 * with that device current, so make that first call before any stream capture.
 */
cg_status cg_solve_noalloc(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                           const double* vals, const double* b, double* x, double tol,
                           int32_t maxit, int32_t precond, void* cuda_stream,
                           int32_t* iters_out, double* relres_out);

#ifdef __cplusplus
}
#endif

#endif /* LIBCG_H */
