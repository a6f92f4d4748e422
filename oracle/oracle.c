/*
 * CG ORACLE — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, sequential, fp64 restatement of what the sparse conjugate-gradient
 * hot path computes, used to check the CUDA library.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header or constant with the CUDA path; both sides only consume the
 * same generated inputs (cgproblems).
 *
 * Paper: "A Preliminary Study on Simultaneous Coscheduling for Discrete GPU
 * vs. Fused GPU" (ICPP Workshops '26).
 *   - CSR SpMV q_i = sum_j A_ij p_j                  Sec. 3.1, equation after Alg. 1
 *   - CG iteration (SpMV, p.q, x/r update, r.r, p)   Alg. 1
 *   - all values, vectors and reductions in fp64     Sec. 3.1
 *   - residual recomputed from the final solution    Sec. 3.1 (last paragraph)
 * Readings where the paper is silent or differs (each also applies to the
 * CUDA path):
 *   R1 relative stopping test ||r||_2 <= tol ||b||_2 instead of the paper's
 *      absolute sqrt(r.r) < tau (Alg. 1 uses b = 1, tau = 1e-8);
 *   R2 the test is made on the recursive residual before the SpMV of each
 *      iteration, so "iterations" counts the SpMVs of the loop;
 *   R3 after the recursive test passes, the true residual b - A x is
 *      recomputed; if it misses tol the solve restarts from the current x
 *      (residual replacement) at most max_restarts times;
 *   R4 p.q <= 0 is a breakdown, a non-finite p.q or rho is a numeric error;
 *   R5 Jacobi preconditioning (not in the paper): z_i = r_i * dinv_i with
 *      dinv_i = 1 / A_ii, p = z + beta p, rho = r.z.  With M = I it is Alg. 1.
 *   R6 mixed precision (not in the paper): textbook iterative refinement,
 *      fp64 true residual and x += d, inner fp32 Jacobi-PCG with fp32
 *      vectors, fp64-accumulated dot products, alpha/beta formed in fp64 and
 *      rounded to fp32 for the fp32 vector updates.
 *   R8 reliable updates (not in the paper; Sleijpen & van der Vorst 1996,
 *      the mixed-precision form of Clark et al. 2010): R6 with the search
 *      direction carried over each fp64 update.  The inner solve of each
 *      outer step ends on its last direction p_k (no update after the last
 *      step) and remembers rho_k = r.z before that step; the next inner solve
 *      starts from the replaced residual r' with p = z' + (r'.z' / rho_k) p_k
 *      instead of p = z', so the Krylov information is not thrown away.
 * Sums run in index order.  Compiled with -ffp-contract=off so no fused
 * multiply-add changes the rounding.
 *
 * The row and vector loops of the fp64 SpMV and (Jacobi-)PCG carry OpenMP
 * row-split pragmas, the form of the paper's CPU runs (Sec. 3.3).  The
 * checker build (no -fopenmp) ignores them and stays sequential, in index
 * order; a second build with -fopenmp exists only to time the same loops on
 * all host cores (its reductions then sum per thread, so its rounding differs
 * and it is never used to check results).
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_NOT_CONVERGED = 1, OR_ERR_INVALID = -1, OR_ERR_BREAKDOWN = -2,
       OR_ERR_NUMERIC = -3, OR_ERR_OOM = -6 };

typedef struct {
  int32_t status;
  int32_t iters;        /* SpMVs inside the loop (R2); total inner iterations for IR */
  int32_t restarts;     /* residual replacements (R3); outer refinement steps for IR */
  int32_t pad;
  double relres_rec;    /* ||r_recursive|| / ||b|| at exit */
  double relres_true;   /* ||b - A x|| / ||b|| recomputed from x (fp64) */
} or_result;

/* y = A x, row by row, terms in storage order (Sec. 3.1) */
void or_spmv(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
             const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += vals[k] * x[colind[k]];
    y[i] = s;
  }
}

double or_dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Threads the row loops use: 1 in the checker build. */
int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ||b - A x||_2 / ||b||_2, 0 when b = 0 (Sec. 3.1, recomputed residual) */
double or_true_relres(int64_t n, const int32_t* rowptr, const int32_t* colind,
                      const double* vals, const double* b, const double* x) {
  double rr = 0.0, bb = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rr, bb)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += vals[k] * x[colind[k]];
    double r = b[i] - s;
    rr += r * r;
    bb += b[i] * b[i];
  }
  return bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
}

/* dinv_i = 1 / A_ii; returns -1 if a diagonal is missing or not positive */
int or_jacobi_dinv(int64_t n, const int32_t* rowptr, const int32_t* colind,
                   const double* vals, double* dinv) {
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    int found = 0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (colind[k] == i) { d += vals[k]; found = 1; }
    if (!found || !(d > 0.0)) return -1;
    dinv[i] = 1.0 / d;
  }
  return 0;
}

/*
 * (Jacobi-preconditioned) CG, Alg. 1 with readings R1-R5.
 *   x        in: x0, out: solution
 *   precond  0 = none (Alg. 1 as printed), 1 = Jacobi (R5)
 *   p_hist   optional [p_hist_k][n]: the first p_hist_k search directions
 *   res_hist optional [maxit+1]: ||r_recursive||/||b|| before each test
 */
int or_pcg(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
           const double* b, double* x, double tol, int32_t maxit, int32_t precond,
           int32_t max_restarts, double* p_hist, int32_t p_hist_k, double* res_hist,
           or_result* out) {
  memset(out, 0, sizeof(*out));
  if (n < 0 || maxit < 0 || !(tol >= 0.0) || (precond != 0 && precond != 1)) {
    out->status = OR_ERR_INVALID;
    return out->status;
  }
  const double bb = or_dot(n, b, b);
  if (bb == 0.0) { /* b = 0: the solution is x = 0 */
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    out->status = OR_OK;
    return OR_OK;
  }
  const double bnorm = sqrt(bb);
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* dinv = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!r || !z || !p || !q || !dinv) {
    free(r); free(z); free(p); free(q); free(dinv);
    out->status = OR_ERR_OOM;
    return out->status;
  }
  if (precond == 1 && or_jacobi_dinv(n, rowptr, colind, vals, dinv) != 0) {
    free(r); free(z); free(p); free(q); free(dinv);
    out->status = OR_ERR_INVALID;
    return out->status;
  }
  int32_t k = 0, restarts = 0, hist = 0, status = OR_NOT_CONVERGED;
  double rr = 0.0;
  for (;;) {
    /* r = b - A x, z = M^-1 r, p = z, rho = r.z */
    or_spmv(n, rowptr, colind, vals, x, q);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) z[i] = precond ? r[i] * dinv[i] : r[i];
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = or_dot(n, r, z);
    rr = or_dot(n, r, r);
    int stop = 0;
    for (;;) {
      if (res_hist) res_hist[k] = sqrt(rr) / bnorm;
      if (sqrt(rr) <= tol * bnorm) break; /* R1, R2 */
      if (k >= maxit) break;
      if (p_hist && hist < p_hist_k) memcpy(p_hist + (size_t)hist++ * (size_t)n, p, sizeof(double) * (size_t)n);
      or_spmv(n, rowptr, colind, vals, p, q); /* q = A p */
      const double pq = or_dot(n, p, q);
      if (!isfinite(pq) || !isfinite(rho)) { status = OR_ERR_NUMERIC; stop = 1; break; }
      if (pq <= 0.0) { status = OR_ERR_BREAKDOWN; stop = 1; break; } /* R4 */
      const double alpha = rho / pq;
      #pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
      #pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
      #pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) z[i] = precond ? r[i] * dinv[i] : r[i];
      const double rho_new = or_dot(n, r, z);
      rr = or_dot(n, r, r);
      const double beta = rho_new / rho;
      rho = rho_new;
      #pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      ++k;
    }
    if (stop) break;
    out->relres_true = or_true_relres(n, rowptr, colind, vals, b, x); /* R3 */
    if (!isfinite(out->relres_true)) { status = OR_ERR_NUMERIC; break; }
    if (out->relres_true <= tol) { status = OR_OK; break; }
    if (k >= maxit || restarts >= max_restarts) { status = OR_NOT_CONVERGED; break; }
    ++restarts;
  }
  out->relres_rec = sqrt(rr) / bnorm;
  if (status == OR_ERR_NUMERIC || status == OR_ERR_BREAKDOWN)
    out->relres_true = or_true_relres(n, rowptr, colind, vals, b, x);
  out->iters = k;
  out->restarts = restarts;
  out->status = status;
  free(r); free(z); free(p); free(q); free(dinv);
  return status;
}

/*
 * Inner fp32 Jacobi-PCG of the refinement (R6): solves A32 d = r32 from d = 0
 * until ||r_d|| <= tol_in ||r32|| or maxit iterations.  Vectors and matrix in
 * fp32; dot products accumulate in fp64; alpha and beta are formed in fp64
 * and rounded to fp32.  Returns the iteration count; *status_out gets
 * OR_OK / OR_NOT_CONVERGED / OR_ERR_BREAKDOWN / OR_ERR_NUMERIC.
 */
static int32_t pcg32(int64_t n, const int32_t* rowptr, const int32_t* colind,
                     const float* vals32, const float* dinv32, const float* rhs, float* d,
                     double tol_in, int32_t maxit, int32_t precond, float* r, float* z,
                     float* p, float* q, int32_t* status_out, int carry, double* rho_io) {
  double bb = 0.0;
  for (int64_t i = 0; i < n; ++i) bb += (double)rhs[i] * (double)rhs[i];
  for (int64_t i = 0; i < n; ++i) { d[i] = 0.0f; r[i] = rhs[i]; }
  for (int64_t i = 0; i < n; ++i) z[i] = precond ? r[i] * dinv32[i] : r[i];
  double rho = 0.0, rr = bb;
  for (int64_t i = 0; i < n; ++i) rho += (double)r[i] * (double)z[i];
  if (carry && *rho_io > 0.0) { /* R8: keep the last direction */
    const float beta0 = (float)(rho / *rho_io);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta0 * p[i];
  } else {
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
  }
  *rho_io = rho;
  int32_t k = 0;
  *status_out = OR_NOT_CONVERGED;
  if (sqrt(rr) <= tol_in * sqrt(bb)) { *status_out = OR_OK; return k; }
  for (;;) {
    if (k >= maxit) break;
    for (int64_t i = 0; i < n; ++i) {
      float s = 0.0f;
      for (int64_t kk = rowptr[i]; kk < rowptr[i + 1]; ++kk) s += vals32[kk] * p[colind[kk]];
      q[i] = s;
    }
    double pq = 0.0;
    for (int64_t i = 0; i < n; ++i) pq += (double)p[i] * (double)q[i];
    if (!isfinite(pq) || !isfinite(rho)) { *status_out = OR_ERR_NUMERIC; break; }
    if (pq <= 0.0) { *status_out = OR_ERR_BREAKDOWN; break; }
    const float alpha = (float)(rho / pq);
    for (int64_t i = 0; i < n; ++i) d[i] += alpha * p[i];
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    for (int64_t i = 0; i < n; ++i) z[i] = precond ? r[i] * dinv32[i] : r[i];
    double rho_new = 0.0;
    rr = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      rho_new += (double)r[i] * (double)z[i];
      rr += (double)r[i] * (double)r[i];
    }
    ++k;
    *rho_io = rho; /* rho_k of the step just taken */
    if (sqrt(rr) <= tol_in * sqrt(bb)) { *status_out = OR_OK; break; }
    if (k >= maxit) break; /* p stays the last direction */
    const float beta = (float)(rho_new / rho);
    rho = rho_new;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  return k;
}

/*
 * fp32-inner / fp64-outer iterative refinement (R6; Higham, "Accuracy and
 * Stability of Numerical Algorithms", ch. 12):
 *   loop: r = b - A x (fp64); stop if ||r||/||b|| <= tol;
 *         solve A32 d = fl32(r) by fp32 Jacobi-PCG to tol_in; x += fl64(d).
 * maxit caps the total inner iterations, max_outer the refinement steps.
 * out->iters = total inner iterations, out->restarts = refinement steps,
 * outer_hist (optional, [max_outer+1]) = ||r||/||b|| at each outer test.
 */
static int pcg_refine(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
                      const double* b, double* x, double tol, double tol_in, int32_t maxit,
                      int32_t max_outer, int32_t precond, double* outer_hist, or_result* out,
                      int carry) {
  memset(out, 0, sizeof(*out));
  if (n < 0 || maxit < 0 || max_outer < 0 || !(tol >= 0.0) || !(tol_in > 0.0) ||
      (precond != 0 && precond != 1)) {
    out->status = OR_ERR_INVALID;
    return out->status;
  }
  const double bb = or_dot(n, b, b);
  if (bb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    out->status = OR_OK;
    return OR_OK;
  }
  const int64_t nnz = rowptr[n];
  const size_t nv = (size_t)(n > 0 ? n : 1);
  double* r = (double*)malloc(sizeof(double) * nv);
  double* dinv = (double*)malloc(sizeof(double) * nv);
  float* vals32 = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
  float* f[7];
  int ok = r && dinv && vals32;
  for (int i = 0; i < 7; ++i) { f[i] = (float*)malloc(sizeof(float) * nv); ok = ok && f[i]; }
  if (!ok) {
    free(r); free(dinv); free(vals32);
    for (int i = 0; i < 7; ++i) free(f[i]);
    out->status = OR_ERR_OOM;
    return out->status;
  }
  float *dinv32 = f[0], *r32 = f[1], *d = f[2], *rr32 = f[3], *z = f[4], *p = f[5], *q = f[6];
  int status = OR_NOT_CONVERGED;
  if (precond == 1 && or_jacobi_dinv(n, rowptr, colind, vals, dinv) != 0) {
    status = OR_ERR_INVALID;
  } else {
    for (int64_t k = 0; k < nnz; ++k) vals32[k] = (float)vals[k];
    for (int64_t i = 0; i < n; ++i) dinv32[i] = precond ? (float)dinv[i] : 1.0f;
    const double bnorm = sqrt(bb);
    int32_t inner_total = 0, outer = 0;
    double relres = 0.0, rho_carry = 0.0;
    for (;;) {
      or_spmv(n, rowptr, colind, vals, x, r);
      double rr = 0.0;
      for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - r[i]; rr += r[i] * r[i]; }
      relres = sqrt(rr) / bnorm;
      if (outer_hist) outer_hist[outer] = relres;
      if (!isfinite(relres)) { status = OR_ERR_NUMERIC; break; }
      if (relres <= tol) { status = OR_OK; break; }
      if (outer >= max_outer || inner_total >= maxit) { status = OR_NOT_CONVERGED; break; }
      for (int64_t i = 0; i < n; ++i) r32[i] = (float)r[i];
      int32_t st;
      inner_total += pcg32(n, rowptr, colind, vals32, dinv32, r32, d, tol_in, maxit - inner_total,
                           precond, rr32, z, p, q, &st, carry, &rho_carry);
      if (st == OR_ERR_NUMERIC || st == OR_ERR_BREAKDOWN) { status = st; break; }
      for (int64_t i = 0; i < n; ++i) x[i] += (double)d[i];
      ++outer;
    }
    out->iters = inner_total;
    out->restarts = outer;
    out->relres_rec = relres;
    out->relres_true = or_true_relres(n, rowptr, colind, vals, b, x);
  }
  out->status = status;
  free(r); free(dinv); free(vals32);
  for (int i = 0; i < 7; ++i) free(f[i]);
  return status;
}

int or_pcg_ir(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
              const double* b, double* x, double tol, double tol_in, int32_t maxit,
              int32_t max_outer, int32_t precond, double* outer_hist, or_result* out) {
  return pcg_refine(n, rowptr, colind, vals, b, x, tol, tol_in, maxit, max_outer, precond,
                    outer_hist, out, 0);
}

/* R8: the refinement with the search direction carried over each fp64 update. */
int or_pcg_ru(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
              const double* b, double* x, double tol, double tol_in, int32_t maxit,
              int32_t max_updates, int32_t precond, double* outer_hist, or_result* out) {
  return pcg_refine(n, rowptr, colind, vals, b, x, tol, tol_in, maxit, max_updates, precond,
                    outer_hist, out, 1);
}

/*
 * ---------------------------------------------------------------------------
 * Factorized sparse approximate inverse preconditioner M^-1 = G^T G
 * (Kolotilina & Yeremin 1993; not in the paper, project-defined).  G is lower
 * triangular in CSR form (grp, gci, gval; columns ascending, the diagonal
 * entry last in each row).  Applying it: t = G r (row sums in storage
 * order), z = G^T t (z_j accumulates G_ij t_i for i ascending).
 * R7 (reading): the PCG with this preconditioner is Alg. 1 with z = G^T G r
 * and rho = r.z, under the same R1-R4 rules as or_pcg.
 */
static void fsai_apply(int64_t n, const int32_t* grp, const int32_t* gci, const double* gval,
                       const double* r, double* t, double* z) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = grp[i]; k < grp[i + 1]; ++k) s += gval[k] * r[gci[k]];
    t[i] = s;
  }
  for (int64_t j = 0; j < n; ++j) z[j] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = grp[i]; k < grp[i + 1]; ++k) z[gci[k]] += gval[k] * t[i];
}

/* PCG with M^-1 = G^T G (R7); *rz_min gets the smallest r.z of the run. */
int or_pcg_fsai(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
                const int32_t* grp, const int32_t* gci, const double* gval, const double* b,
                double* x, double tol, int32_t maxit, int32_t max_restarts, double* res_hist,
                double* rz_min, or_result* out) {
  memset(out, 0, sizeof(*out));
  if (n < 0 || maxit < 0 || !(tol >= 0.0)) {
    out->status = OR_ERR_INVALID;
    return out->status;
  }
  const double bb = or_dot(n, b, b);
  if (rz_min) *rz_min = INFINITY;
  if (bb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    out->status = OR_OK;
    return OR_OK;
  }
  const double bnorm = sqrt(bb);
  const size_t nv = (size_t)(n > 0 ? n : 1);
  double* r = (double*)malloc(sizeof(double) * nv);
  double* z = (double*)malloc(sizeof(double) * nv);
  double* p = (double*)malloc(sizeof(double) * nv);
  double* q = (double*)malloc(sizeof(double) * nv);
  double* t = (double*)malloc(sizeof(double) * nv);
  if (!r || !z || !p || !q || !t) {
    free(r); free(z); free(p); free(q); free(t);
    out->status = OR_ERR_OOM;
    return out->status;
  }
  int32_t k = 0, restarts = 0, status = OR_NOT_CONVERGED;
  double rr = 0.0;
  for (;;) {
    or_spmv(n, rowptr, colind, vals, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    fsai_apply(n, grp, gci, gval, r, t, z);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = or_dot(n, r, z);
    rr = or_dot(n, r, r);
    int stop = 0;
    for (;;) {
      if (rz_min && rho < *rz_min) *rz_min = rho;
      if (res_hist) res_hist[k] = sqrt(rr) / bnorm;
      if (sqrt(rr) <= tol * bnorm) break;
      if (k >= maxit) break;
      or_spmv(n, rowptr, colind, vals, p, q);
      const double pq = or_dot(n, p, q);
      if (!isfinite(pq) || !isfinite(rho)) { status = OR_ERR_NUMERIC; stop = 1; break; }
      if (pq <= 0.0) { status = OR_ERR_BREAKDOWN; stop = 1; break; }
      const double alpha = rho / pq;
      for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
      for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
      fsai_apply(n, grp, gci, gval, r, t, z);
      const double rho_new = or_dot(n, r, z);
      rr = or_dot(n, r, r);
      const double beta = rho_new / rho;
      rho = rho_new;
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      ++k;
    }
    if (stop) break;
    out->relres_true = or_true_relres(n, rowptr, colind, vals, b, x);
    if (!isfinite(out->relres_true)) { status = OR_ERR_NUMERIC; break; }
    if (out->relres_true <= tol) { status = OR_OK; break; }
    if (k >= maxit || restarts >= max_restarts) { status = OR_NOT_CONVERGED; break; }
    ++restarts;
  }
  out->relres_rec = sqrt(rr) / bnorm;
  if (status == OR_ERR_NUMERIC || status == OR_ERR_BREAKDOWN)
    out->relres_true = or_true_relres(n, rowptr, colind, vals, b, x);
  out->iters = k;
  out->restarts = restarts;
  out->status = status;
  free(r); free(z); free(p); free(q); free(t);
  return status;
}

/* fp32 G^T G application: t = G r, z = G^T t with fp32 values and sums. */
static void fsai_apply32(int64_t n, const int32_t* grp, const int32_t* gci, const float* g32,
                         const float* r, float* t, float* z) {
  for (int64_t i = 0; i < n; ++i) {
    float s = 0.0f;
    for (int64_t k = grp[i]; k < grp[i + 1]; ++k) s += g32[k] * r[gci[k]];
    t[i] = s;
  }
  for (int64_t j = 0; j < n; ++j) z[j] = 0.0f;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = grp[i]; k < grp[i + 1]; ++k) z[gci[k]] += g32[k] * t[i];
}

/* Inner fp32 PCG of the refinement with M^-1 = G32^T G32 (R6 with R7). */
static int32_t pcg32_fsai(int64_t n, const int32_t* rowptr, const int32_t* colind,
                          const float* vals32, const int32_t* grp, const int32_t* gci,
                          const float* g32, const float* rhs, float* d, double tol_in,
                          int32_t maxit, float* r, float* z, float* p, float* q, float* t,
                          int32_t* status_out, int carry, double* rho_io) {
  double bb = 0.0;
  for (int64_t i = 0; i < n; ++i) bb += (double)rhs[i] * (double)rhs[i];
  for (int64_t i = 0; i < n; ++i) { d[i] = 0.0f; r[i] = rhs[i]; }
  fsai_apply32(n, grp, gci, g32, r, t, z);
  double rho = 0.0, rr = bb;
  for (int64_t i = 0; i < n; ++i) rho += (double)r[i] * (double)z[i];
  if (carry && *rho_io > 0.0) { /* R8 */
    const float beta0 = (float)(rho / *rho_io);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta0 * p[i];
  } else {
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
  }
  *rho_io = rho;
  int32_t k = 0;
  *status_out = OR_NOT_CONVERGED;
  if (sqrt(rr) <= tol_in * sqrt(bb)) { *status_out = OR_OK; return k; }
  for (;;) {
    if (k >= maxit) break;
    for (int64_t i = 0; i < n; ++i) {
      float s = 0.0f;
      for (int64_t kk = rowptr[i]; kk < rowptr[i + 1]; ++kk) s += vals32[kk] * p[colind[kk]];
      q[i] = s;
    }
    double pq = 0.0;
    for (int64_t i = 0; i < n; ++i) pq += (double)p[i] * (double)q[i];
    if (!isfinite(pq) || !isfinite(rho)) { *status_out = OR_ERR_NUMERIC; break; }
    if (pq <= 0.0) { *status_out = OR_ERR_BREAKDOWN; break; }
    const float alpha = (float)(rho / pq);
    for (int64_t i = 0; i < n; ++i) d[i] += alpha * p[i];
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    fsai_apply32(n, grp, gci, g32, r, t, z);
    double rho_new = 0.0;
    rr = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      rho_new += (double)r[i] * (double)z[i];
      rr += (double)r[i] * (double)r[i];
    }
    ++k;
    *rho_io = rho;
    if (sqrt(rr) <= tol_in * sqrt(bb)) { *status_out = OR_OK; break; }
    if (k >= maxit) break;
    const float beta = (float)(rho_new / rho);
    rho = rho_new;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  return k;
}

/* fp32-inner / fp64-outer refinement (R6) whose inner PCG uses M^-1 = G^T G (R7). */
static int fsai_refine(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
                       const int32_t* grp, const int32_t* gci, const double* gval, const double* b,
                       double* x, double tol, double tol_in, int32_t maxit, int32_t max_outer,
                       double* outer_hist, or_result* out, int carry) {
  memset(out, 0, sizeof(*out));
  if (n < 0 || maxit < 0 || max_outer < 0 || !(tol >= 0.0) || !(tol_in > 0.0)) {
    out->status = OR_ERR_INVALID;
    return out->status;
  }
  const double bb = or_dot(n, b, b);
  if (bb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    out->status = OR_OK;
    return OR_OK;
  }
  const int64_t nnz = rowptr[n], gnnz = grp[n];
  const size_t nv = (size_t)(n > 0 ? n : 1);
  double* r = (double*)malloc(sizeof(double) * nv);
  float* vals32 = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
  float* g32 = (float*)malloc(sizeof(float) * (size_t)(gnnz > 0 ? gnnz : 1));
  float* f[7];
  int ok = r && vals32 && g32;
  for (int i = 0; i < 7; ++i) { f[i] = (float*)malloc(sizeof(float) * nv); ok = ok && f[i]; }
  if (!ok) {
    free(r); free(vals32); free(g32);
    for (int i = 0; i < 7; ++i) free(f[i]);
    out->status = OR_ERR_OOM;
    return out->status;
  }
  float *r32 = f[0], *d = f[1], *rw = f[2], *z = f[3], *p = f[4], *q = f[5], *t = f[6];
  for (int64_t k = 0; k < nnz; ++k) vals32[k] = (float)vals[k];
  for (int64_t k = 0; k < gnnz; ++k) g32[k] = (float)gval[k];
  const double bnorm = sqrt(bb);
  int32_t inner_total = 0, outer = 0, status = OR_NOT_CONVERGED;
  double relres = 0.0, rho_carry = 0.0;
  for (;;) {
    or_spmv(n, rowptr, colind, vals, x, r);
    double rr = 0.0;
    for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - r[i]; rr += r[i] * r[i]; }
    relres = sqrt(rr) / bnorm;
    if (outer_hist) outer_hist[outer] = relres;
    if (!isfinite(relres)) { status = OR_ERR_NUMERIC; break; }
    if (relres <= tol) { status = OR_OK; break; }
    if (outer >= max_outer || inner_total >= maxit) { status = OR_NOT_CONVERGED; break; }
    for (int64_t i = 0; i < n; ++i) r32[i] = (float)r[i];
    int32_t st;
    inner_total += pcg32_fsai(n, rowptr, colind, vals32, grp, gci, g32, r32, d, tol_in,
                              maxit - inner_total, rw, z, p, q, t, &st, carry, &rho_carry);
    if (st == OR_ERR_NUMERIC || st == OR_ERR_BREAKDOWN) { status = st; break; }
    for (int64_t i = 0; i < n; ++i) x[i] += (double)d[i];
    ++outer;
  }
  out->iters = inner_total;
  out->restarts = outer;
  out->relres_rec = relres;
  out->relres_true = or_true_relres(n, rowptr, colind, vals, b, x);
  out->status = status;
  free(r); free(vals32); free(g32);
  for (int i = 0; i < 7; ++i) free(f[i]);
  return status;
}

int or_pcg_ir_fsai(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
                   const int32_t* grp, const int32_t* gci, const double* gval, const double* b,
                   double* x, double tol, double tol_in, int32_t maxit, int32_t max_outer,
                   double* outer_hist, or_result* out) {
  return fsai_refine(n, rowptr, colind, vals, grp, gci, gval, b, x, tol, tol_in, maxit, max_outer,
                     outer_hist, out, 0);
}

/* R8 with M^-1 = G32^T G32 (R7). */
int or_pcg_ru_fsai(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
                   const int32_t* grp, const int32_t* gci, const double* gval, const double* b,
                   double* x, double tol, double tol_in, int32_t maxit, int32_t max_updates,
                   double* outer_hist, or_result* out) {
  return fsai_refine(n, rowptr, colind, vals, grp, gci, gval, b, x, tol, tol_in, maxit,
                     max_updates, outer_hist, out, 1);
}
