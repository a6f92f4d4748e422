// Factorized sparse approximate inverse preconditioning, M^-1 = G^T G
// (Kolotilina & Yeremin 1993; not in the paper): the pattern of G (that of
// tril(A)), the classic factor, user-supplied factors, the factor's ELL
// layouts for the loop, and the persistent PCG kernels that apply it.  The
// learned factor (an MLP over matrix features) lives in cg_mlp.cu.
//
// PCG with G^T G (standard form, Alg. 1 with z = G^T G r):
//   phase 1: q = A p, p.q                                  -> alpha
//   phase 2: r' = r - alpha q (into the other r buffer), r'.r',
//            t = G r' (r' of neighbour rows recomputed from r and q, so no
//            barrier is needed between the r update and G r'), t.t = r'.z,
//            x += alpha p                                  -> beta, test
//   phase 3: p = G^T t + beta p
// Three grid barriers per iteration, as for Jacobi.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "cg_fsai.cuh"
#include "cg_graph.cuh"

using namespace cg;

namespace {

cg_status ffail(cg_handle* h, cg_status s, const std::string& msg) {
  h->err = msg;
  return s;
}

#define CGF_CUDA(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return ffail((h), e_ == cudaErrorMemoryAllocation ? CG_ERR_OOM : CG_ERR_CUDA,        \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

unsigned blocks_for(int64_t items) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 8192));
}

// Classic FSAI (F2), thread per row: the local matrix A[P_i, P_i] (P_i the
// row's tril pattern, ascending, ending with i) is factored by Cholesky and
// A_loc y = e_last solved; g_i = y / sqrt(y_last).  bad[0] counts rows whose
// local matrix is not SPD.
__global__ void classic_fsai_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                    const int32_t* __restrict__ colind, const double* __restrict__ vals,
                                    const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                    double* __restrict__ g, unsigned long long* bad) {
  constexpr int M = kFsaiMaxRow;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t0 = trp[i], m = trp[i + 1] - t0;
    double L[M * (M + 1) / 2];  // packed lower triangle, row a at a (a + 1) / 2
    int P[M];
    for (int a = 0; a < m; ++a) P[a] = tci[t0 + a];
    // A_loc[a][c] for c <= a: merge row P[a] of A with P (both ascending)
    for (int a = 0; a < m; ++a) {
      int c = 0;
      for (int k = rowptr[P[a]]; k < rowptr[P[a] + 1] && c <= a; ++k) {
        const int col = colind[k];
        while (c <= a && P[c] < col) L[a * (a + 1) / 2 + c++] = 0.0;
        if (c <= a && P[c] == col) L[a * (a + 1) / 2 + c++] = vals[k];
      }
      while (c <= a) L[a * (a + 1) / 2 + c++] = 0.0;
    }
    // Cholesky in place
    bool ok = true;
    for (int a = 0; a < m && ok; ++a) {
      for (int c = 0; c <= a; ++c) {
        double s = L[a * (a + 1) / 2 + c];
        for (int k = 0; k < c; ++k) s -= L[a * (a + 1) / 2 + k] * L[c * (c + 1) / 2 + k];
        if (c == a) {
          if (!(s > 0.0)) { ok = false; break; }
          L[a * (a + 1) / 2 + a] = sqrt(s);
        } else {
          L[a * (a + 1) / 2 + c] = s / L[c * (c + 1) / 2 + c];
        }
      }
    }
    if (!ok) {
      atomicAdd(bad, 1ull);
      for (int a = 0; a < m; ++a) g[t0 + a] = 0.0;
      continue;
    }
    // L L^T y = e_last: forward (L w = e_last: w = 0 except w_last), then back
    double y[M];
    for (int a = 0; a < m; ++a) y[a] = 0.0;
    y[m - 1] = 1.0 / L[(m - 1) * m / 2 + (m - 1)];
    for (int a = m - 1; a >= 0; --a) {
      double s = y[a];
      for (int c = a + 1; c < m; ++c) s -= L[c * (c + 1) / 2 + a] * y[c];
      y[a] = s / L[a * (a + 1) / 2 + a];
    }
    const double sc = 1.0 / sqrt(y[m - 1]);
    for (int a = 0; a < m; ++a) g[t0 + a] = y[a] * sc;
  }
}

// ELL layouts of G and G^T for the loop from the factor values (tril order):
// slot m of row i at [m n + i]; src = tril index or -1 (padding: the row's own
// column, value 0).
template <typename T>
__global__ void fill_ell_kernel(int64_t n, int w, const int32_t* __restrict__ src, const double* __restrict__ g,
                                T* __restrict__ val) {
  const int64_t total = (int64_t)w * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int s = src[e];
    val[e] = s >= 0 ? (T)g[s] : T(0);
  }
}

// Diagonal layouts of G and G^T: entry e = (i, j) of tril(A) in slot s_e of
// row i of G and in slot nd - 1 - s_e of row j of G^T (the offsets of G^T are
// those of G negated, in reverse order).  Every position is written at most
// once; the rest stays 0 from the memset.
template <typename T>
__global__ void fill_dia_kernel(int64_t nt, int64_t n, int nd, const int32_t* __restrict__ trow,
                                const int32_t* __restrict__ tci, const int8_t* __restrict__ slot,
                                const double* __restrict__ g, T* __restrict__ gv, T* __restrict__ gtv) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = slot[e];
    gv[(int64_t)s * n + trow[e]] = (T)g[e];
    gtv[(int64_t)(nd - 1 - s) * n + tci[e]] = (T)g[e];
  }
}

__global__ void g_positive_kernel(int64_t n, const int32_t* __restrict__ trp, const double* __restrict__ g,
                                  unsigned long long* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = g[trp[i + 1] - 1];  // the diagonal ends the row
    if (!(d > 0.0) || !isfinite(d)) atomicAdd(bad, 1ull);
  }
}

// ---------------------------------------------------------------- the PCG loop

// G or G^T for the loop: slot m of row i at [m n + i]; the column is col[m n + i]
// (ELL) or, in the diagonal layout (DIA), i + delta[m] clamped into [0, n) (the
// value is 0 wherever the diagonal leaves the pattern).
template <typename T>
struct Ell {
  const int32_t* col;
  const T* val;
  int w;
  int delta[kFsaiMaxDiag];
};

template <bool DIA, typename T>
__device__ __forceinline__ int ell_col(const Ell<T>& E, int m, int64_t i, int64_t n) {
  if (DIA) return min(max((int)i + E.delta[m], 0), (int)n - 1);
  return __ldg(E.col + m * n + i);
}

template <typename T>
struct FsaiVecs {
  T *r0, *r1, *p, *q, *t, *x;  // x: the iterate (fp64) or the correction d (refinement)
};

struct FsaiParams {
  SolveParams P;            // A (CSR and loop matrix, unscaled), b, x, partials, limits
  Ell<double> G64, GT64;
  Ell<float> G32, GT32;
  FsaiVecs<double> V64;
  FsaiVecs<float> V32;
};

// t = G r (r the current residual), rho = t.t = r.z; then p = G^T t, or with
// rho_prev > 0 (reliable updates, R8) p = G^T t + (rho / rho_prev) p.
template <bool DIA, typename T>
__device__ bool fsai_start(const Ell<T>& G, const Ell<T>& GT, const FsaiVecs<T>& V, const T* r, int64_t n,
                           double* part, int pstride, Grid& g, double* rho, double rho_prev = 0.0) {
  Acc<T> a;
  for (int64_t i = g.gtid; i < n; i += g.gstride) {
    T s = T(0);
    for (int m = 0; m < G.w; ++m) s = fma(__ldg(G.val + m * n + i), r[ell_col<DIA>(G, m, i, n)], s);
    V.t[i] = s;
    a.add(s, s);
  }
  double v[1] = {a.get()};
  publish<1>(v, part + kSlotRes * (size_t)pstride, g);
  if (!g.sync()) return false;
  grid_sum<1>(part + kSlotRes * (size_t)pstride, g.G, v);
  *rho = v[0];
  const bool carry = rho_prev > 0.0;
  const T beta = carry ? (T)(v[0] / rho_prev) : T(0);
  for (int64_t i = g.gtid; i < n; i += g.gstride) {
    T s = T(0);
    for (int m = 0; m < GT.w; ++m) s = fma(__ldg(GT.val + m * n + i), V.t[ell_col<DIA>(GT, m, i, n)], s);
    V.p[i] = carry ? fma(beta, V.p[i], s) : s;
  }
  return g.sync();
}

// The PCG loop from a start state (r in V.r0, p = G^T G r, rho = r.z, rr =
// r.r) until sqrt(rr) <= stop_abs (kOk), maxit (kNotConverged), breakdown /
// non-finite values, or a barrier timeout.  x += alpha p each iteration.
template <bool DIA, typename T>
__device__ int fsai_loop(const Sell<T>& S, const Ell<T>& G, const Ell<T>& GT, const FsaiVecs<T>& V, double rho,
                         double rr, double stop_abs, int maxit, int* iters, double* part, int pstride, Grid& g,
                         double* rho_last = nullptr) {
  const int64_t n = S.n;
  if (rho_last) *rho_last = rho;
  int k = *iters;
  int status = kNotConverged;
  if (sqrt(rr) <= stop_abs) status = kOk;
  bool done = sqrt(rr) <= stop_abs || k >= maxit;
  T* rc = V.r0;
  T* rn = V.r1;
  while (!done) {
    double v1[1] = {spmv_phase<T, false>(S, V.p, V.q, g)};
    publish<1>(v1, part + kSlotPQ * (size_t)pstride, g);
    if (!g.sync()) { status = kTimeout; break; }
    double pq[1];
    grid_sum<1>(part + kSlotPQ * (size_t)pstride, g.G, pq);
    if (!isfinite(pq[0]) || !isfinite(rho)) { status = kNumeric; break; }
    if (pq[0] <= 0.0) { status = kBreakdown; break; }
    const T alpha = (T)(rho / pq[0]);
    Acc<T> a_rho, a_rr;
    for (int64_t i = g.gtid; i < n; i += g.gstride) {
      const T ri = fma(-alpha, V.q[i], rc[i]);
      rn[i] = ri;
      a_rr.add(ri, ri);
      T s = T(0);
      for (int m = 0; m < G.w; ++m) {
        const int j = ell_col<DIA>(G, m, i, n);
        s = fma(__ldg(G.val + m * n + i), fma(-alpha, V.q[j], rc[j]), s);
      }
      V.t[i] = s;
      a_rho.add(s, s);
      V.x[i] = fma(alpha, V.p[i], V.x[i]);
    }
    double v2[2] = {a_rho.get(), a_rr.get()};
    publish<2>(v2, part + kSlotUpd * (size_t)pstride, g);
    if (!g.sync()) { status = kTimeout; break; }
    double s2[2];
    grid_sum<2>(part + kSlotUpd * (size_t)pstride, g.G, s2);
    const T beta = (T)(s2[0] / rho);
    if (rho_last) *rho_last = rho;
    rho = s2[0];
    rr = s2[1];
    ++k;
    const bool conv = sqrt(rr) <= stop_abs;
    done = conv || k >= maxit;
    if (conv) status = kOk;
    T* tmp = rc;
    rc = rn;
    rn = tmp;
    if (!done) {
      for (int64_t i = g.gtid; i < n; i += g.gstride) {
        T s = T(0);
        for (int m = 0; m < GT.w; ++m) s = fma(__ldg(GT.val + m * n + i), V.t[ell_col<DIA>(GT, m, i, n)], s);
        V.p[i] = fma(beta, V.p[i], s);
      }
      if (!g.sync()) { status = kTimeout; break; }
    }
  }
  *iters = k;
  return status;
}

// fp64 PCG with G^T G: true-residual check and restarts as cg_solve (R1-R5, R7).
template <bool DIA>
__global__ void __launch_bounds__(kBlock, 2) pcg_fsai64_kernel(FsaiParams F) {
  __shared__ double s_prod[kCap];
  const SolveParams& P = F.P;
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  const int64_t n = P.A.n;
  const FsaiVecs<double>& V = F.V64;
  int status = kNotConverged, k = 0, restarts = 0;
  double relres_true = 0.0, bb = 0.0;
  bool first = true;
  for (;;) {
    spmv_orig(P.A, P.x, V.q, g, s_prod);
    if (!g.sync()) { status = kTimeout; break; }
    double v[2] = {0.0, 0.0};
    for (int64_t i = g.gtid; i < n; i += g.gstride) {
      const double bi = P.b[i];
      const double ri = bi - V.q[i];
      V.r0[i] = ri;
      v[0] += ri * ri;
      v[1] += bi * bi;
    }
    publish<2>(v, P.part + kSlotRes * (size_t)P.pstride, g);
    if (!g.sync()) { status = kTimeout; break; }
    double s2[2];
    grid_sum<2>(P.part + kSlotRes * (size_t)P.pstride, g.G, s2);
    const double rr_start = s2[0];
    if (first) {
      bb = s2[1];
      if (bb == 0.0) {
        for (int64_t i = g.gtid; i < n; i += g.gstride) P.x[i] = 0.0;
        status = kOk;
        break;
      }
    }
    relres_true = sqrt(rr_start) / sqrt(bb);
    if (!first) {
      if (!isfinite(relres_true)) { status = kNumeric; break; }
      if (relres_true <= P.tol) { status = kOk; break; }
      if (k >= P.maxit || restarts >= P.max_restarts) { status = kNotConverged; break; }
      ++restarts;
    } else if (sqrt(rr_start) <= P.tol * sqrt(bb)) {
      status = kOk;  // x0 meets tol
      break;
    } else if (k >= P.maxit) {
      status = kNotConverged;
      break;
    }
    first = false;
    double rho = 0.0;
    if (!fsai_start<DIA, double>(F.G64, F.GT64, V, V.r0, n, P.part, P.pstride, g, &rho)) { status = kTimeout; break; }
    const int st = fsai_loop<DIA, double>(P.S64, F.G64, F.GT64, V, rho, rr_start, P.tol * sqrt(bb), P.maxit, &k,
                                     P.part, P.pstride, g);
    if (st == kTimeout) { status = kTimeout; break; }
    if (st == kNumeric || st == kBreakdown) {
      status = st;
      spmv_orig(P.A, P.x, V.q, g, s_prod);  // the true residual of the last iterate
      if (!g.sync()) { status = kTimeout; break; }
      double w[1] = {0.0};
      for (int64_t i = g.gtid; i < n; i += g.gstride) {
        const double ri = P.b[i] - V.q[i];
        w[0] += ri * ri;
      }
      publish<1>(w, P.part + kSlotRes * (size_t)P.pstride, g);
      if (!g.sync()) { status = kTimeout; break; }
      grid_sum<1>(P.part + kSlotRes * (size_t)P.pstride, g.G, w);
      relres_true = sqrt(w[0]) / sqrt(bb);
      break;
    }
    // kOk or kNotConverged: back to the true residual
  }
  if (g.cta == 0 && threadIdx.x == 0) {
    P.st->status = status;
    P.st->iters = k;
    P.st->restarts = restarts;
    P.st->relres_true = relres_true;
    P.st->relres_rec = relres_true;
  }
}

// fp32-inner / fp64-outer refinement (R6) with the inner M^-1 = G32^T G32 (R7);
// CARRY: reliable updates (R8), the search direction survives each fp64 update.
template <bool DIA, bool CARRY>
__global__ void __launch_bounds__(kBlock, 2) pcg_fsai_ir_kernel(FsaiParams F) {
  __shared__ double s_prod[kCap];
  const SolveParams& P = F.P;
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  const int64_t n = P.A.n;
  const FsaiVecs<float>& V = F.V32;
  int status = kNotConverged, inner = 0, outer = 0;
  double relres = 0.0, bb = 0.0, rho_k = 0.0;
  for (;;) {
    spmv_orig(P.A, P.x, F.V64.q, g, s_prod);
    if (!g.sync()) { status = kTimeout; break; }
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t i = g.gtid; i < n; i += g.gstride) {
      const double bi = P.b[i];
      const double ri = bi - F.V64.q[i];
      const float r32 = (float)ri;
      V.r0[i] = r32;
      V.x[i] = 0.0f;
      v[0] += ri * ri;
      v[1] += bi * bi;
      v[2] += (double)r32 * (double)r32;
    }
    publish<3>(v, P.part + kSlotRes * (size_t)P.pstride, g);
    if (!g.sync()) { status = kTimeout; break; }
    double s3[3];
    grid_sum<3>(P.part + kSlotRes * (size_t)P.pstride, g.G, s3);
    if (outer == 0) {
      bb = s3[1];
      if (bb == 0.0) {
        for (int64_t i = g.gtid; i < n; i += g.gstride) P.x[i] = 0.0;
        status = kOk;
        break;
      }
    }
    relres = sqrt(s3[0]) / sqrt(bb);
    if (!isfinite(relres)) { status = kNumeric; break; }
    if (relres <= P.tol) { status = kOk; break; }
    if (outer >= P.max_restarts || inner >= P.maxit) { status = kNotConverged; break; }
    double rho = 0.0;
    if (!fsai_start<DIA, float>(F.G32, F.GT32, V, V.r0, n, P.part, P.pstride, g, &rho,
                                CARRY && outer > 0 ? rho_k : 0.0)) { status = kTimeout; break; }
    const int st = fsai_loop<DIA, float>(P.S32, F.G32, F.GT32, V, rho, s3[2], P.tol_in * sqrt(s3[2]), P.maxit, &inner,
                                    P.part, P.pstride, g, &rho_k);
    if (st == kTimeout || st == kNumeric || st == kBreakdown) { status = st; break; }
    for (int64_t i = g.gtid; i < n; i += g.gstride) P.x[i] += (double)V.x[i];
    if (!g.sync()) { status = kTimeout; break; }
    ++outer;
  }
  if (g.cta == 0 && threadIdx.x == 0) {
    P.st->status = status;
    P.st->iters = inner;
    P.st->restarts = outer;
    P.st->relres_true = relres;
    P.st->relres_rec = relres;
  }
}


// ---------------------------------------------------------------- graph form
// The fp32 refinement loop with G^T G as CUDA graph nodes (large systems):
//   outer WHILE { q64 = A x | r32 = fl32(b - q64), d = 0 | t = G r32 |
//                 start (1 CTA: fp64 test, limits, carry factor) | p = G^T t (+ beta0 p) |
//                 inner WHILE { q = A p, p.q | alpha, r', t = G r', d += alpha p |
//                               beta, test, p = G^T t + beta p or x64 += d } }
// Every phase is its own kernel (the kernel boundaries are the barriers); each
// CTA re-forms the scalars from the fixed-order partials of the previous kernel.
constexpr int kSlotT = kSlotRes + 3;  // t.t of the start pass
constexpr int64_t kFsaiGraphMinRows = 1 << 19;  // auto loop form: graph from here (fp32 inner)

struct FArgs {
  GArgs a;
  Ell<float> G, GT;
  float* r[2];  // current residual in r[k & 1]
  float* t;
  float* d;     // the inner solve's correction
  int carry;    // reliable updates (R8)
};

__global__ void __launch_bounds__(kBlock) gf_res(FArgs F) {
  const SolveParams& P = F.a.P;
  Grid g = graph_grid();
  float* r = F.r[F.a.gs->k & 1];
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = g.gtid; i < P.A.n; i += g.gstride) {
    const double bi = P.b[i];
    const double ri = bi - P.V64.q[i];
    const float r32 = (float)ri;
    r[i] = r32;
    F.d[i] = 0.0f;
    v[0] += ri * ri;
    v[1] += bi * bi;
    v[2] += (double)r32 * (double)r32;
  }
  publish<3>(v, P.part + kSlotRes * (size_t)P.pstride, g);
}

template <bool DIA>
__global__ void __launch_bounds__(kBlock) gf_t(FArgs F) {
  const SolveParams& P = F.a.P;
  Grid g = graph_grid();
  const int64_t n = P.A.n;
  const float* r = F.r[F.a.gs->k & 1];
  Acc<float> a;
  for (int64_t i = g.gtid; i < n; i += g.gstride) {
    float s = 0.0f;
    for (int m = 0; m < F.G.w; ++m) s = fmaf(__ldg(F.G.val + m * n + i), r[ell_col<DIA>(F.G, m, i, n)], s);
    F.t[i] = s;
    a.add(s, s);
  }
  double v[1] = {a.get()};
  publish<1>(v, P.part + kSlotT * (size_t)P.pstride, g);
}

// One CTA: the fp64 residual test and limits; the next inner solve's state.
template <bool COND>
__global__ void gf_start(FArgs F) {
  const SolveParams& P = F.a.P;
  double s[3], tt[1];
  grid_sum<3>(P.part + kSlotRes * (size_t)P.pstride, F.a.G_upd, s);
  grid_sum<1>(P.part + kSlotT * (size_t)P.pstride, F.a.G_upd, tt);
  if (threadIdx.x != 0) return;
  GState* gs = F.a.gs;
  if (!gs->started) {
    gs->started = 1;
    gs->bb = s[1];
    gs->k = 0;
    gs->outer = 0;
    gs->status = kRunning;
    gs->rho_k = 0.0;
  }
  const double rel = gs->bb > 0.0 ? sqrt(s[0]) / sqrt(gs->bb) : 0.0;
  gs->relres_true = rel;
  bool stop = true;
  int status = gs->status;
  if (status == kBreakdown || status == kNumeric) {
    // the previous inner solve failed; x keeps the last good iterate
  } else if (gs->bb == 0.0) {
    status = kOk;
  } else if (!isfinite(rel)) {
    status = kNumeric;
  } else if (rel <= P.tol) {
    status = kOk;
  } else if (gs->outer >= P.max_restarts || gs->k >= P.maxit) {
    status = kNotConverged;
  } else {
    stop = false;
  }
  bool inner = false;
  if (!stop) {
    gs->beta0 = (F.carry && gs->outer > 0 && gs->rho_k > 0.0) ? tt[0] / gs->rho_k : 0.0;
    gs->rho = tt[0];
    gs->rho_k = tt[0];
    gs->rr = s[2];
    gs->stop_abs = P.tol_in * sqrt(s[2]);
    gs->k_start = gs->k;
    gs->outer += 1;
    gs->ctr = 0;
    status = kRunning;
    inner = !(sqrt(s[2]) <= gs->stop_abs);
  }
  gs->status = status;
  if constexpr (COND) {
    cudaGraphSetConditional(F.a.h2, stop ? 0u : 1u);
    cudaGraphSetConditional(F.a.h, inner ? 1u : 0u);
  }
}

// p = G^T t, or p = G^T t + beta0 p when the direction is carried over.
template <bool DIA>
__global__ void __launch_bounds__(kBlock) gf_p0(FArgs F) {
  const SolveParams& P = F.a.P;
  if (F.a.gs->status != kRunning) return;
  Grid g = graph_grid();
  const int64_t n = P.A.n;
  const float beta0 = (float)F.a.gs->beta0;
  float* p = P.V32.p;
  for (int64_t i = g.gtid; i < n; i += g.gstride) {
    float s = 0.0f;
    for (int m = 0; m < F.GT.w; ++m) s = fmaf(__ldg(F.GT.val + m * n + i), F.t[ell_col<DIA>(F.GT, m, i, n)], s);
    p[i] = beta0 != 0.0f ? fmaf(beta0, p[i], s) : s;
  }
}

template <bool DIA>
__global__ void __launch_bounds__(kBlock) gf_upd_r(FArgs F) {
  const SolveParams& P = F.a.P;
  GState* gs = F.a.gs;
  if (gs->status != kRunning) return;
  Grid g = graph_grid();
  const int64_t n = P.A.n;
  double pq[1];
  grid_sum<1>(P.part + kSlotPQ * (size_t)P.pstride, F.a.G_spmv, pq);
  __shared__ double s_alpha;
  __shared__ int s_stop;
  if (threadIdx.x == 0) {  // scalars once per CTA
    const double rho = gs->rho;
    const int st = (!isfinite(pq[0]) || !isfinite(rho)) ? kNumeric : (pq[0] <= 0.0 ? kBreakdown : 0);
    if (st && g.cta == 0) gs->status = st;
    s_stop = st;
    s_alpha = rho / pq[0];
  }
  __syncthreads();
  if (s_stop) return;
  const float alpha = (float)s_alpha;
  const int k = gs->k;
  const float* rc = F.r[k & 1];
  float* rn = F.r[(k + 1) & 1];
  const float* q = P.V32.q;
  const float* p = P.V32.p;
  Acc<float> a_rho, a_rr;
  for (int64_t i = g.gtid; i < n; i += g.gstride) {
    const float ri = fmaf(-alpha, q[i], rc[i]);
    rn[i] = ri;
    a_rr.add(ri, ri);
    float s = 0.0f;
    for (int m = 0; m < F.G.w; ++m) {
      const int j = ell_col<DIA>(F.G, m, i, n);
      s = fmaf(__ldg(F.G.val + m * n + i), fmaf(-alpha, q[j], rc[j]), s);
    }
    F.t[i] = s;
    a_rho.add(s, s);
    F.d[i] = fmaf(alpha, p[i], F.d[i]);
  }
  double v[2] = {a_rho.get(), a_rr.get()};
  publish<2>(v, P.part + kSlotUpd * (size_t)P.pstride, g);
}

template <bool DIA, bool COND>
__global__ void __launch_bounds__(kBlock) gf_upd_p(FArgs F) {
  const SolveParams& P = F.a.P;
  GState* gs = F.a.gs;
  Grid g = graph_grid();
  const int64_t n = P.A.n;
  const bool failed = gs->status != kRunning;
  double s2[2] = {0.0, 0.0};
  __shared__ double s_beta;
  __shared__ int s_fl;  // done | conv << 1
  const int k1 = gs->k + 1;
  if (!failed) {
    grid_sum<2>(P.part + kSlotUpd * (size_t)P.pstride, F.a.G_upd, s2);
    if (threadIdx.x == 0) {
      s_beta = s2[0] / gs->rho;
      const bool conv = sqrt(s2[1]) <= gs->stop_abs;
      s_fl = (conv || k1 >= P.maxit ? 1 : 0) | (conv ? 2 : 0);
    }
    __syncthreads();
    if (!(s_fl & 1)) {
      const float beta = (float)s_beta;
      float* p = P.V32.p;
      for (int64_t i = g.gtid; i < n; i += g.gstride) {
        float s = 0.0f;
        for (int m = 0; m < F.GT.w; ++m) s = fmaf(__ldg(F.GT.val + m * n + i), F.t[ell_col<DIA>(F.GT, m, i, n)], s);
        p[i] = fmaf(beta, p[i], s);
      }
    } else {
      for (int64_t i = g.gtid; i < n; i += g.gstride) P.x[i] += (double)F.d[i];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&gs->ctr, 1u) == g.G - 1) {  // every CTA has read the state and finished
      gs->ctr = 0;
      const bool done = failed || (s_fl & 1);
      if (!failed) {
        gs->rho_k = gs->rho;
        gs->rho = s2[0];
        gs->rr = s2[1];
        gs->k = k1;
        gs->status = (s_fl & 1) ? ((s_fl & 2) ? kOk : kNotConverged) : kRunning;
      }
      __threadfence();
      if constexpr (COND) cudaGraphSetConditional(F.a.h, done ? 0u : 1u);
    }
  }
}

cudaError_t add_node(cudaGraph_t g, cudaGraphNode_t* node, cudaGraphNode_t dep, const void* fn, unsigned grid,
                     unsigned block, void** args) {
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
}

cg_status build_fsai_graph(cg_handle* h, const FArgs& Fin);

cg_status solve_fsai_graph(cg_handle* h, const FArgs& F, bool carry, int32_t* iters_out, double* relres_out) {
  FsaiData* f = h->fsai;
  const SolveParams& P = F.a.P;
  if (!f->gexec || f->gkey_b != P.b || f->gkey_x != P.x || f->gkey_tol != P.tol || f->gkey_maxit != P.maxit ||
      f->gkey_tol_in != P.tol_in || f->gkey_outer != P.max_restarts || f->gkey_carry != (int)carry ||
      f->gkey_kind != f->dia) {
    const cg_status s = build_fsai_graph(h, F);
    if (s != CG_OK) return s;
    f->gkey_b = P.b;
    f->gkey_x = P.x;
    f->gkey_tol = P.tol;
    f->gkey_maxit = P.maxit;
    f->gkey_tol_in = P.tol_in;
    f->gkey_outer = P.max_restarts;
    f->gkey_carry = carry;
    f->gkey_kind = f->dia;
  }
  CGF_CUDA(h, cudaMemsetAsync(h->gs, 0, sizeof(GState), h->stream));
  CGF_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  CGF_CUDA(h, cudaGraphLaunch(f->gexec, h->stream));
  CGF_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  CGF_CUDA(h, cudaMemcpyAsync(h->host_gs, h->gs, sizeof(GState), cudaMemcpyDeviceToHost, h->stream));
  CGF_CUDA(h, cudaStreamSynchronize(h->stream));
  float ms = 0.0f;
  CGF_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  const GState& gs = *h->host_gs;
  const int status = gs.status;
  const int64_t n = h->n;
  h->last.status = status;
  h->last.iters = gs.k;
  h->last.restarts = gs.outer;
  h->last.grid_ctas = h->grid_graph;
  h->last.relres_true = gs.relres_true;
  h->last.relres_rec = gs.relres_true;
  h->last.kernel_ms = ms;
  h->last.loop_form = 2;
  h->last.kernel_launches = (int32_t)std::min<int64_t>(5 * (int64_t)(gs.outer + 1) + 3 * (int64_t)gs.k + 1, INT32_MAX);
  h->last.precond_used = CG_PRECOND_FSAI;
  const int64_t per_iter = 8 * (h->nnz + 2 * f->ntril) + 4 * (n + 1) + 13 * 4 * n;
  h->last.bytes_moved = per_iter * (int64_t)gs.k;
  h->last.kernel_bytes_per_iter = per_iter;
  if (iters_out) *iters_out = gs.k;
  if (relres_out) *relres_out = gs.relres_true;
  if (status < 0) return ffail(h, (cg_status)status, std::string("cg_solve (FSAI): ") + cg_status_string(status));
  return (cg_status)status;
}


void destroy_fsai_graph(FsaiData* f) {
  if (f->gexec) cudaGraphExecDestroy(f->gexec);
  if (f->graph) cudaGraphDestroy(f->graph);
  f->gexec = nullptr;
  f->graph = nullptr;
}

cg_status build_fsai_graph(cg_handle* h, const FArgs& Fin) {
  FsaiData* f = h->fsai;
  destroy_fsai_graph(f);
  cudaGraph_t g;
  CGF_CUDA(h, cudaGraphCreate(&g, 0));
  f->graph = g;
  cudaGraphConditionalHandle outer_h, inner_h;
  CGF_CUDA(h, cudaGraphConditionalHandleCreate(&outer_h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams op{};
  op.type = cudaGraphNodeTypeConditional;
  op.conditional.handle = outer_h;
  op.conditional.type = cudaGraphCondTypeWhile;
  op.conditional.size = 1;
  cudaGraphNode_t on;
  CGF_CUDA(h, cudaGraphAddNode(&on, g, nullptr, nullptr, 0, &op));
  cudaGraph_t ob = op.conditional.phGraph_out[0];
  CGF_CUDA(h, cudaGraphConditionalHandleCreate(&inner_h, ob, 0, cudaGraphCondAssignDefault));
  FArgs F = Fin;
  F.a.h = inner_h;
  F.a.h2 = outer_h;
  const void* f_spmv = cgi::spmv_kernel_f32(h);
  int per_sm = 0;
  CGF_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f_spmv, kBlock, 0));
  const unsigned G = (unsigned)h->grid_graph;
  const unsigned Gq = (unsigned)std::max(1, std::min(per_sm * h->sm_count, h->grid_part));
  F.a.G_spmv = Gq;
  F.a.G_upd = G;
  // kernel arguments are copied into the nodes at creation
  Csr<double> A = F.a.P.A;
  const double* gx = F.a.P.x;
  double* gq = F.a.P.V64.q;
  void* a_spmv[] = {&A, &gx, &gq};
  void* a_f[] = {&F};
  void* a_ga[] = {&F.a};
  const unsigned Gs = (unsigned)std::min<int64_t>(std::max<int32_t>(h->nrb, 1), (int64_t)h->sm_count * 64);
  const bool dia = f->dia != 0;
  cudaGraphNode_t n, prev;
  CGF_CUDA(h, add_node(ob, &n, nullptr, (const void*)spmv_kernel<double>, Gs, kBlock, a_spmv));
  prev = n;
  CGF_CUDA(h, add_node(ob, &n, prev, (const void*)gf_res, G, kBlock, a_f));
  prev = n;
  CGF_CUDA(h, add_node(ob, &n, prev, dia ? (const void*)gf_t<true> : (const void*)gf_t<false>, G, kBlock, a_f));
  prev = n;
  CGF_CUDA(h, add_node(ob, &n, prev, (const void*)gf_start<true>, 1, 32, a_f));
  prev = n;
  CGF_CUDA(h, add_node(ob, &n, prev, dia ? (const void*)gf_p0<true> : (const void*)gf_p0<false>, G, kBlock, a_f));
  prev = n;
  cudaGraphNodeParams ip{};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = inner_h;
  ip.conditional.type = cudaGraphCondTypeWhile;
  ip.conditional.size = 1;
  CGF_CUDA(h, cudaGraphAddNode(&n, ob, &prev, nullptr, 1, &ip));
  cudaGraph_t ib = ip.conditional.phGraph_out[0];
  cudaGraphNode_t b1, b2, b3;
  CGF_CUDA(h, add_node(ib, &b1, nullptr, f_spmv, Gq, kBlock, a_ga));
  CGF_CUDA(h, add_node(ib, &b2, b1, dia ? (const void*)gf_upd_r<true> : (const void*)gf_upd_r<false>, G, kBlock,
                       a_f));
  CGF_CUDA(h, add_node(ib, &b3, b2, dia ? (const void*)gf_upd_p<true, true> : (const void*)gf_upd_p<false, true>, G,
                       kBlock, a_f));
  CGF_CUDA(h, add_node(g, &n, on, (const void*)g_flush_ir, G, kBlock, a_ga));
  CGF_CUDA(h, cudaGraphInstantiate(&f->gexec, g, 0));
  return CG_OK;
}

}  // namespace

void cgi::fsai_free(FsaiData* f) {
  if (!f) return;
  void* dev[] = {f->trp,   f->tci,    f->tsrc,   f->g,      f->gsrc,  f->gcol,  f->gval64, f->gval32,
                 f->gtsrc, f->gtcol,  f->gtval64, f->gtval32, f->r0,   f->r1,    f->t,      f->r0_32,
                 f->r1_32, f->t_32,   f->x_32,   f->offs,   f->work,  f->dout,  f->gpart,  f->mlp_o,
                 f->params32, f->trow, f->rpart, f->tslot};
  for (void* p : dev)
    if (p) cudaFree(p);
  destroy_fsai_graph(f);
  delete f;
}

// Pattern of G (tril(A)) and of G^T, their ELL slot maps, once per handle.
cg_status cgi::fsai_pattern(cg_handle* h) {
  if (h->fsai) return CG_OK;
  if (!h->jacobi_ok) return ffail(h, CG_ERR_INVALID, "FSAI needs a positive diagonal in every row");
  const int64_t n = h->n, nnz = h->nnz;
  std::vector<int32_t> ci((size_t)nnz);
  if (nnz > 0)
    CGF_CUDA(h, cudaMemcpy(ci.data(), h->colind, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost));
  const std::vector<int32_t>& rp = h->host_rowptr;
  std::vector<int32_t> trp((size_t)n + 1, 0), tci, tsrc;
  tci.reserve((size_t)(nnz / 2 + n));
  tsrc.reserve((size_t)(nnz / 2 + n));
  for (int64_t i = 0; i < n; ++i) {
    int last = -1;
    for (int k = rp[(size_t)i]; k < rp[(size_t)i + 1]; ++k) {
      const int c = ci[(size_t)k];
      if (c <= last) return ffail(h, CG_ERR_INVALID, "FSAI needs strictly increasing columns in each row");
      last = c;
      if (c <= i) {
        tci.push_back(c);
        tsrc.push_back(k);
      }
    }
    trp[(size_t)i + 1] = (int32_t)tci.size();
    const int len = trp[(size_t)i + 1] - trp[(size_t)i];
    if (len == 0 || tci.back() != i) return ffail(h, CG_ERR_INVALID, "FSAI needs a diagonal entry in every row");
    if (len > kFsaiMaxRow)
      return ffail(h, CG_ERR_INVALID, "FSAI: a row of tril(A) has more than " + std::to_string(kFsaiMaxRow) +
                                          " entries");
  }
  const int64_t nt = (int64_t)tci.size();
  // G^T rows: entries (i, j) of tril grouped by column j, i ascending
  std::vector<int32_t> cnt((size_t)n, 0);
  for (int64_t e = 0; e < nt; ++e) ++cnt[(size_t)tci[(size_t)e]];
  int gw = 0, gtw = 0;
  for (int64_t i = 0; i < n; ++i) {
    gw = std::max(gw, trp[(size_t)i + 1] - trp[(size_t)i]);
    gtw = std::max(gtw, cnt[(size_t)i]);
  }
  if (gtw > kFsaiMaxCol)
    return ffail(h, CG_ERR_INVALID, "FSAI: a column of tril(A) has more than " + std::to_string(kFsaiMaxCol) +
                                        " entries");
  std::vector<int32_t> gsrc((size_t)gw * n), gcol((size_t)gw * n), gtsrc((size_t)gtw * n), gtcol((size_t)gtw * n);
  for (int64_t i = 0; i < n; ++i) {
    const int a = trp[(size_t)i], len = trp[(size_t)i + 1] - a;
    for (int m = 0; m < gw; ++m) {
      gsrc[(size_t)m * n + i] = m < len ? a + m : -1;
      gcol[(size_t)m * n + i] = m < len ? tci[(size_t)(a + m)] : (int32_t)i;
    }
  }
  std::vector<int32_t> fillc((size_t)n, 0);
  for (int64_t i = 0; i < n; ++i)  // rows ascending: G^T row j lists i ascending
    for (int e = trp[(size_t)i]; e < trp[(size_t)i + 1]; ++e) {
      const int j = tci[(size_t)e];
      const int m = fillc[(size_t)j]++;
      gtsrc[(size_t)m * n + j] = e;
      gtcol[(size_t)m * n + j] = (int32_t)i;
    }
  for (int64_t j = 0; j < n; ++j)
    for (int m = fillc[(size_t)j]; m < gtw; ++m) {
      gtsrc[(size_t)m * n + j] = -1;
      gtcol[(size_t)m * n + j] = (int32_t)j;
    }
  // diagonal layout when tril(A) lies on at most kFsaiMaxDiag offsets
  std::vector<int32_t> toffs;
  std::vector<int32_t> trow((size_t)nt);
  for (int64_t i = 0; i < n; ++i)
    for (int e = trp[(size_t)i]; e < trp[(size_t)i + 1]; ++e) {
      trow[(size_t)e] = (int32_t)i;
      const int o = tci[(size_t)e] - (int)i;
      if ((int)toffs.size() <= kFsaiMaxDiag && std::find(toffs.begin(), toffs.end(), o) == toffs.end())
        toffs.push_back(o);
    }
  const bool dia = (int)toffs.size() <= kFsaiMaxDiag;
  std::vector<int8_t> tslot;
  if (dia) {
    std::sort(toffs.begin(), toffs.end());
    tslot.resize((size_t)nt);
    for (int64_t e = 0; e < nt; ++e) {
      const int o = tci[(size_t)e] - trow[(size_t)e];
      tslot[(size_t)e] = (int8_t)(std::lower_bound(toffs.begin(), toffs.end(), o) - toffs.begin());
    }
  }
  FsaiData* f = new FsaiData();
  h->fsai = f;
  f->ntril = nt;
  f->gw = gw;
  f->gtw = gtw;
  f->dia = dia ? 1 : 0;
  f->nd = dia ? (int)toffs.size() : 0;
  for (int m = 0; m < f->nd; ++m) f->doff[m] = toffs[(size_t)m];
  auto up = [&](int32_t** d, const std::vector<int32_t>& v) -> cudaError_t {
    cudaError_t e = cudaMalloc(d, sizeof(int32_t) * std::max<size_t>(v.size(), 1));
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*d, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice);
    return e;
  };
  CGF_CUDA(h, up(&f->trp, trp));
  CGF_CUDA(h, up(&f->tci, tci));
  CGF_CUDA(h, up(&f->tsrc, tsrc));
  CGF_CUDA(h, up(&f->gsrc, gsrc));
  CGF_CUDA(h, up(&f->gcol, gcol));
  CGF_CUDA(h, up(&f->gtsrc, gtsrc));
  CGF_CUDA(h, up(&f->gtcol, gtcol));
  CGF_CUDA(h, up(&f->trow, trow));
  if (dia) {
    CGF_CUDA(h, cudaMalloc(&f->tslot, std::max<size_t>(tslot.size(), 1)));
    if (nt > 0) CGF_CUDA(h, cudaMemcpy(f->tslot, tslot.data(), tslot.size(), cudaMemcpyHostToDevice));
  }
  const size_t nv = (size_t)std::max<int64_t>(n, 1);
  gw = std::max(gw, f->nd);  // value arrays serve either layout
  gtw = std::max(gtw, f->nd);
  CGF_CUDA(h, cudaMalloc(&f->g, sizeof(double) * (size_t)std::max<int64_t>(nt, 1)));
  CGF_CUDA(h, cudaMalloc(&f->gval64, sizeof(double) * (size_t)gw * nv));
  CGF_CUDA(h, cudaMalloc(&f->gval32, sizeof(float) * (size_t)gw * nv));
  CGF_CUDA(h, cudaMalloc(&f->gtval64, sizeof(double) * (size_t)gtw * nv));
  CGF_CUDA(h, cudaMalloc(&f->gtval32, sizeof(float) * (size_t)gtw * nv));
  for (double** v : {&f->r0, &f->r1, &f->t}) CGF_CUDA(h, cudaMalloc(v, sizeof(double) * nv));
  for (float** v : {&f->r0_32, &f->r1_32, &f->t_32, &f->x_32}) CGF_CUDA(h, cudaMalloc(v, sizeof(float) * nv));
  return CG_OK;
}

// Check the factor in f->g (positive diagonal) and refresh the loop's ELL values.
cg_status cgi::fsai_commit(cg_handle* h, int kind) {
  FsaiData* f = h->fsai;
  const int64_t n = h->n;
  unsigned long long* bad = nullptr;
  CGF_CUDA(h, cudaMalloc(&bad, sizeof(unsigned long long)));
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) {
    g_positive_kernel<<<blocks_for(n), 256, 0, h->stream>>>(n, f->trp, f->g, bad);
    e = cudaGetLastError();
  }
  unsigned long long hb = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(bad);
  CGF_CUDA(h, e);
  if (hb) {
    f->kind = 0;
    return ffail(h, CG_ERR_INVALID, "FSAI factor: " + std::to_string(hb) + " rows without a positive finite diagonal");
  }
  if (f->dia) {
    const size_t w = (size_t)f->nd * (size_t)n;
    CGF_CUDA(h, cudaMemsetAsync(f->gval64, 0, sizeof(double) * w, h->stream));
    CGF_CUDA(h, cudaMemsetAsync(f->gtval64, 0, sizeof(double) * w, h->stream));
    CGF_CUDA(h, cudaMemsetAsync(f->gval32, 0, sizeof(float) * w, h->stream));
    CGF_CUDA(h, cudaMemsetAsync(f->gtval32, 0, sizeof(float) * w, h->stream));
    fill_dia_kernel<double><<<blocks_for(f->ntril), 256, 0, h->stream>>>(f->ntril, n, f->nd, f->trow, f->tci,
                                                                         f->tslot, f->g, f->gval64, f->gtval64);
    fill_dia_kernel<float><<<blocks_for(f->ntril), 256, 0, h->stream>>>(f->ntril, n, f->nd, f->trow, f->tci,
                                                                        f->tslot, f->g, f->gval32, f->gtval32);
  } else {
    fill_ell_kernel<double><<<blocks_for((int64_t)f->gw * n), 256, 0, h->stream>>>(n, f->gw, f->gsrc, f->g, f->gval64);
    fill_ell_kernel<float><<<blocks_for((int64_t)f->gw * n), 256, 0, h->stream>>>(n, f->gw, f->gsrc, f->g, f->gval32);
    fill_ell_kernel<double><<<blocks_for((int64_t)f->gtw * n), 256, 0, h->stream>>>(n, f->gtw, f->gtsrc, f->g,
                                                                                    f->gtval64);
    fill_ell_kernel<float><<<blocks_for((int64_t)f->gtw * n), 256, 0, h->stream>>>(n, f->gtw, f->gtsrc, f->g,
                                                                                   f->gtval32);
  }
  CGF_CUDA(h, cudaGetLastError());
  CGF_CUDA(h, cudaStreamSynchronize(h->stream));
  f->kind = kind;
  return CG_OK;
}

// The PCG with the handle's factor; P carries the unscaled loop matrices.
cg_status cgi::fsai_solve(cg_handle* h, const SolveParams& Pin, bool fp64, bool carry, int grid,
                          int32_t* iters_out, double* relres_out) {
  FsaiData* f = h->fsai;
  const int64_t n = h->n;
  FsaiParams F{};
  F.P = Pin;
  const int w = f->dia ? f->nd : f->gw, wt = f->dia ? f->nd : f->gtw;
  F.G64 = Ell<double>{f->gcol, f->gval64, w, {}};
  F.GT64 = Ell<double>{f->gtcol, f->gtval64, wt, {}};
  F.G32 = Ell<float>{f->gcol, f->gval32, w, {}};
  F.GT32 = Ell<float>{f->gtcol, f->gtval32, wt, {}};
  for (int m = 0; m < (f->dia ? f->nd : 0); ++m) {
    F.G64.delta[m] = F.G32.delta[m] = f->doff[m];
    F.GT64.delta[m] = F.GT32.delta[m] = -f->doff[f->nd - 1 - m];
  }
  F.V64 = FsaiVecs<double>{f->r0, f->r1, Pin.V64.p, Pin.V64.q, f->t, Pin.x};
  F.V32 = FsaiVecs<float>{f->r0_32, f->r1_32, Pin.V32.p, Pin.V32.q, f->t_32, f->x_32};
  if (!fp64 && (h->loop_mode == 2 || (h->loop_mode == 0 && n >= kFsaiGraphMinRows))) {
    FArgs FA{};
    FA.a.P = Pin;
    FA.a.gs = h->gs;
    FA.G = F.G32;
    FA.GT = F.GT32;
    FA.r[0] = f->r0_32;
    FA.r[1] = f->r1_32;
    FA.t = f->t_32;
    FA.d = f->x_32;
    FA.carry = carry ? 1 : 0;
    return solve_fsai_graph(h, FA, carry, iters_out, relres_out);
  }
  void* args[] = {&F};
  const void* fn;
  if (fp64) fn = f->dia ? (const void*)pcg_fsai64_kernel<true> : (const void*)pcg_fsai64_kernel<false>;
  else if (carry) fn = f->dia ? (const void*)pcg_fsai_ir_kernel<true, true> : (const void*)pcg_fsai_ir_kernel<false, true>;
  else fn = f->dia ? (const void*)pcg_fsai_ir_kernel<true, false> : (const void*)pcg_fsai_ir_kernel<false, false>;
  int per_sm = 0;
  CGF_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0));
  const int G = std::max(1, std::min(grid, per_sm * h->sm_count));
  CGF_CUDA(h, cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream));
  CGF_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  CGF_CUDA(h, cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kBlock), args, 0, h->stream));
  CGF_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  CGF_CUDA(h, cudaMemcpyAsync(h->host_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CGF_CUDA(h, cudaStreamSynchronize(h->stream));
  float ms = 0.0f;
  CGF_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  const DevState& ds = *h->host_st;
  const cg_status status = ds.abort ? CG_ERR_TIMEOUT : (cg_status)ds.status;
  h->last.status = status;
  h->last.iters = ds.iters;
  h->last.restarts = ds.restarts;
  h->last.grid_ctas = G;
  h->last.relres_true = ds.relres_true;
  h->last.relres_rec = ds.relres_rec;
  h->last.kernel_ms = ms;
  h->last.loop_form = 1;
  h->last.kernel_launches = 1;
  h->last.precond_used = CG_PRECOND_FSAI;
  // modelled bytes per iteration: A (CSR), G and G^T (values + columns) and the vector streams
  const int64_t vb = fp64 ? 8 : 4, ib = 4;
  const int64_t per_iter = (vb + ib) * (h->nnz + 2 * f->ntril) + 4 * (n + 1) + 13 * vb * n;
  h->last.loop_form = 1;
  h->last.bytes_moved = per_iter * (int64_t)ds.iters;
  h->last.kernel_bytes_per_iter = per_iter;
  if (iters_out) *iters_out = ds.iters;
  if (relres_out) *relres_out = ds.relres_true;
  if (status == CG_ERR_TIMEOUT) return ffail(h, status, "cg_solve (FSAI): a grid barrier timed out");
  if (status < 0) return ffail(h, status, std::string("cg_solve (FSAI): ") + cg_status_string(status));
  return status;
}

extern "C" {

cg_status cg_fsai_classic(cg_handle* h) {
  if (!h) return CG_ERR_INVALID;
  if (h->batch) return ffail(h, CG_ERR_INVALID, "cg_fsai_classic: batch handle");
  if (h->n == 0) return ffail(h, CG_ERR_INVALID, "cg_fsai_classic: empty matrix");
  cg_status s = cgi::fsai_pattern(h);
  if (s != CG_OK) return s;
  FsaiData* f = h->fsai;
  unsigned long long* bad = nullptr;
  CGF_CUDA(h, cudaMalloc(&bad, sizeof(unsigned long long)));
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) {
    classic_fsai_kernel<<<blocks_for(h->n), 128, 0, h->stream>>>(h->n, h->rowptr, h->colind, h->vals, f->trp,
                                                                  f->tci, f->g, bad);
    e = cudaGetLastError();
  }
  unsigned long long hb = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(bad);
  CGF_CUDA(h, e);
  if (hb) {
    f->kind = 0;
    return ffail(h, CG_ERR_INVALID, "cg_fsai_classic: " + std::to_string(hb) + " local matrices are not SPD");
  }
  return cgi::fsai_commit(h, 1);
}

cg_status cg_fsai_set_factor(cg_handle* h, const double* g_tril) {
  if (!h) return CG_ERR_INVALID;
  if (h->batch) return ffail(h, CG_ERR_INVALID, "cg_fsai_set_factor: batch handle");
  if (!g_tril || h->n == 0) return ffail(h, CG_ERR_INVALID, "cg_fsai_set_factor: NULL values or empty matrix");
  cg_status s = cgi::fsai_pattern(h);
  if (s != CG_OK) return s;
  CGF_CUDA(h, cudaMemcpyAsync(h->fsai->g, g_tril, sizeof(double) * (size_t)h->fsai->ntril, cudaMemcpyDeviceToDevice,
                              h->stream));
  return cgi::fsai_commit(h, 3);
}

cg_status cg_fsai_get_factor(cg_handle* h, double* g_tril, int64_t* ntril, int32_t* kind) {
  if (!h) return CG_ERR_INVALID;
  if (h->batch) return ffail(h, CG_ERR_INVALID, "cg_fsai_get_factor: batch handle");
  if (h->n > 0 && !h->fsai) {
    cg_status s = cgi::fsai_pattern(h);
    if (s != CG_OK) return s;
  }
  const FsaiData* f = h->fsai;
  if (ntril) *ntril = f ? f->ntril : 0;
  if (kind) *kind = f ? f->kind : 0;
  if (g_tril && f && f->kind) {
    CGF_CUDA(h, cudaMemcpyAsync(g_tril, f->g, sizeof(double) * (size_t)f->ntril, cudaMemcpyDeviceToDevice,
                                h->stream));
    CGF_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return CG_OK;
}

}  // extern "C"
