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


// Slot form of G and G^T in the loop kernels (template parameter W): kEll =
// column arrays, kDiaAny = diagonal layout with a run-time slot count, W > 0 =
// diagonal layout with exactly W slots (the common stencil widths: 3 for a
// 2-D 5-point, 4 for a 3-D 7-point, 5 for a 2-D 9-point or Q1 pattern).
constexpr int kEll = 0, kDiaAny = -1;

// sum_m E(i, m) * f(column of slot m) in slot order.  With W slots known at
// compile time every load of the row is issued before the first product (a
// loop over a run-time count waits a full memory latency per slot).
template <int W, typename T, typename Fn>
__device__ __forceinline__ T ell_row(const Ell<T>& E, int64_t i, int64_t n, Fn&& f) {
  T s = T(0);
  if constexpr (W > 0) {
    T e[W], v[W];
#pragma unroll
    for (int m = 0; m < W; ++m) {
      e[m] = __ldg(E.val + (int64_t)m * n + i);
      v[m] = f(min(max((int)i + E.delta[m], 0), (int)n - 1));
    }
#pragma unroll
    for (int m = 0; m < W; ++m) s = fma(e[m], v[m], s);
  } else if constexpr (W == kDiaAny) {
#pragma unroll
    for (int m = 0; m < kFsaiMaxDiag; ++m)
      if (m < E.w) s = fma(__ldg(E.val + (int64_t)m * n + i), f(min(max((int)i + E.delta[m], 0), (int)n - 1)), s);
  } else {
    for (int m = 0; m < E.w; ++m) s = fma(__ldg(E.val + m * n + i), f(__ldg(E.col + m * n + i)), s);
  }
  return s;
}

// The rows gtid, gtid + gstride, ... of a grid-stride loop, two at a time:
// load(i) reads a row's inputs and forms its results (no stores), store(i, v)
// writes them, in row order.  Both rows' loads are in flight before the first
// store, which the compiler may not move loads across.
template <class Load, class Store>
__device__ __forceinline__ void rows_x2(const Grid& g, int64_t n, Load&& load, Store&& store) {
  int64_t i = g.gtid;
  for (; i + g.gstride < n; i += 2 * g.gstride) {
    const auto a = load(i);
    const auto b = load(i + g.gstride);
    store(i, a);
    store(i + g.gstride, b);
  }
  if (i < n) store(i, load(i));
}

template <typename T>
struct RowUpd {
  T r, t, x;
};

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
template <int W, typename T>
__device__ bool fsai_start(const Ell<T>& G, const Ell<T>& GT, const FsaiVecs<T>& V, const T* r, int64_t n,
                           double* part, int pstride, Grid& g, double* rho, double rho_prev = 0.0) {
  constexpr bool kExact = sizeof(T) == 4;  // the fp64 loop keeps the fp64 sums (register budget)
  Acc<T> a;
  rows_x2(
      g, n, [&](int64_t i) { return ell_row<W>(G, i, n, [&](int j) { return r[j]; }); },
      [&](int64_t i, T s) {
        V.t[i] = s;
        a.add(s, s);
      });
  double v[1] = {a.get()};
  publish<1, kExact>(v, part + kSlotRes * (size_t)pstride, g);
  if (!g.sync()) return false;
  grid_sum<1, kExact>(part + kSlotRes * (size_t)pstride, g.G, v);
  *rho = v[0];
  const bool carry = rho_prev > 0.0;
  const T beta = carry ? (T)(v[0] / rho_prev) : T(0);
  rows_x2(
      g, n,
      [&](int64_t i) {
        const T s = ell_row<W>(GT, i, n, [&](int j) { return V.t[j]; });
        return carry ? fma(beta, V.p[i], s) : s;
      },
      [&](int64_t i, T pi) { V.p[i] = pi; });
  return g.sync();
}

// The PCG loop from a start state (r in V.r0, p = G^T G r, rho = r.z, rr =
// r.r) until sqrt(rr) <= stop_abs (kOk), maxit (kNotConverged), breakdown /
// non-finite values, or a barrier timeout.  x += alpha p each iteration.
template <int W, typename T>
__device__ int fsai_loop(const Sell<T>& S, const Ell<T>& G, const Ell<T>& GT, const FsaiVecs<T>& V, double rho,
                         double rr, double stop_abs, int maxit, int* iters, double* part, int pstride, Grid& g,
                         double* rho_last = nullptr) {
  constexpr bool kExact = sizeof(T) == 4;  // the fp64 loop keeps the fp64 sums (register budget)
  const int64_t n = S.n;
  if (rho_last) *rho_last = rho;
  int k = *iters;
  int status = kNotConverged;
  if (sqrt(rr) <= stop_abs) status = kOk;
  bool done = sqrt(rr) <= stop_abs || k >= maxit;
  const double stop2_hi = stop2_high(stop_abs);
  T* rc = V.r0;
  T* rn = V.r1;
  while (!done) {
    double v1[1] = {spmv_phase<T, false>(S, V.p, V.q, g)};
    publish<1, kExact>(v1, part + kSlotPQ * (size_t)pstride, g);
    if (!g.sync()) { status = kTimeout; break; }
    double pq[1];
    grid_sum<1, kExact>(part + kSlotPQ * (size_t)pstride, g.G, pq);
    // the scalars once per CTA (an fp64 divide or square root in every
    // thread would load GB300's narrow fp64 pipe), shared through shared memory
    __shared__ double s_sc[2];
    __shared__ int s_fl;
    if (threadIdx.x == 0) {
      s_fl = (!isfinite(pq[0]) || !isfinite(rho)) ? kNumeric : (pq[0] <= 0.0 ? kBreakdown : 0);
      s_sc[0] = rho / pq[0];
    }
    __syncthreads();
    if (s_fl) { status = s_fl; break; }
    const T alpha = (T)s_sc[0];
    // 1 / rho for this iteration's beta, in warp 1 during the r update: beta =
    // rho' (1 / rho) is a multiply after the next grid sum (within 1.5 ulp of rho' / rho)
    __shared__ double s_inv_rho;
    if (threadIdx.x == 32) s_inv_rho = 1.0 / rho;
    Acc<T> a_rho, a_rr;
    rows_x2(
        g, n,
        [&](int64_t i) {
          RowUpd<T> u;
          u.r = fma(-alpha, V.q[i], rc[i]);
          u.t = ell_row<W>(G, i, n, [&](int j) { return fma(-alpha, V.q[j], rc[j]); });
          u.x = fma(alpha, V.p[i], V.x[i]);
          return u;
        },
        [&](int64_t i, const RowUpd<T>& u) {
          rn[i] = u.r;
          a_rr.add(u.r, u.r);
          V.t[i] = u.t;
          a_rho.add(u.t, u.t);
          V.x[i] = u.x;
        });
    double v2[2] = {a_rho.get(), a_rr.get()};
    publish<2, kExact>(v2, part + kSlotUpd * (size_t)pstride, g);
    if (!g.sync()) { status = kTimeout; break; }
    double s2[2];
    grid_sum<2, kExact>(part + kSlotUpd * (size_t)pstride, g.G, s2);
    if (threadIdx.x == 0) {
      s_sc[1] = s2[0] * s_inv_rho;
      s_fl = below_stop(s2[1], stop_abs, stop2_hi);
    }
    __syncthreads();
    const T beta = (T)s_sc[1];
    const bool conv = s_fl != 0;
    if (rho_last) *rho_last = rho;
    rho = s2[0];
    rr = s2[1];
    ++k;
    done = conv || k >= maxit;
    if (conv) status = kOk;
    T* tmp = rc;
    rc = rn;
    rn = tmp;
    if (!done) {
      rows_x2(
          g, n, [&](int64_t i) { return fma(beta, V.p[i], ell_row<W>(GT, i, n, [&](int j) { return V.t[j]; })); },
          [&](int64_t i, T pi) { V.p[i] = pi; });
      if (!g.sync()) { status = kTimeout; break; }
    }
  }
  *iters = k;
  return status;
}

// fp64 PCG with G^T G: true-residual check and restarts as cg_solve (R1-R5, R7).
template <int W>
__global__ void __launch_bounds__(kBlock, 2) pcg_fsai64_kernel(FsaiParams F) {
  const SolveParams& P = F.P;
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  const int64_t n = P.A.n;
  const FsaiVecs<double>& V = F.V64;
  int status = kNotConverged, k = 0, restarts = 0;
  double relres_true = 0.0, bb = 0.0;
  bool first = true;
  for (;;) {
    spmv_orig(P.A, P.x, V.q, g);
    if (!g.sync()) { status = kTimeout; break; }
    double v[2] = {0.0, 0.0};
    for (int64_t i = g.gtid; i < n; i += g.gstride) {
      const double bi = P.b[i];
      const double ri = bi - V.q[i];
      V.r0[i] = ri;
      v[0] += ri * ri;
      v[1] += bi * bi;
    }
    publish<2, false>(v, P.part + kSlotRes * (size_t)P.pstride, g);
    if (!g.sync()) { status = kTimeout; break; }
    double s2[2];
    grid_sum<2, false>(P.part + kSlotRes * (size_t)P.pstride, g.G, s2);
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
    if (!fsai_start<W, double>(F.G64, F.GT64, V, V.r0, n, P.part, P.pstride, g, &rho)) { status = kTimeout; break; }
    const int st = fsai_loop<W, double>(P.S64, F.G64, F.GT64, V, rho, rr_start, P.tol * sqrt(bb), P.maxit, &k,
                                     P.part, P.pstride, g);
    if (st == kTimeout) { status = kTimeout; break; }
    if (st == kNumeric || st == kBreakdown) {
      status = st;
      spmv_orig(P.A, P.x, V.q, g);  // the true residual of the last iterate
      if (!g.sync()) { status = kTimeout; break; }
      double w[1] = {0.0};
      for (int64_t i = g.gtid; i < n; i += g.gstride) {
        const double ri = P.b[i] - V.q[i];
        w[0] += ri * ri;
      }
      publish<1, false>(w, P.part + kSlotRes * (size_t)P.pstride, g);
      if (!g.sync()) { status = kTimeout; break; }
      grid_sum<1, false>(P.part + kSlotRes * (size_t)P.pstride, g.G, w);
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
template <int W, bool CARRY>
__global__ void __launch_bounds__(kBlock, 2) pcg_fsai_ir_kernel(FsaiParams F) {
  const SolveParams& P = F.P;
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  const int64_t n = P.A.n;
  const FsaiVecs<float>& V = F.V32;
  int status = kNotConverged, inner = 0, outer = 0;
  double relres = 0.0, bb = 0.0, rho_k = 0.0;
  for (;;) {
    spmv_orig(P.A, P.x, F.V64.q, g);
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
    if (!fsai_start<W, float>(F.G32, F.GT32, V, V.r0, n, P.part, P.pstride, g, &rho,
                                CARRY && outer > 0 ? rho_k : 0.0)) { status = kTimeout; break; }
    const int st = fsai_loop<W, float>(P.S32, F.G32, F.GT32, V, rho, s3[2], P.tol_in * sqrt(s3[2]), P.maxit, &inner,
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
//   outer WHILE { x64 += d (after an inner solve) | q64 = A x | r32 = fl32(b - q64), d = 0 |
//                 t = G r32 | start (1 CTA: fp64 test, limits, carry factor) | p = G^T t (+ beta0 p) |
//                 inner WHILE { q = A p, p.q -> alpha | r', t = G r', d += alpha p -> beta, test |
//                               p = G^T t + beta p } }
// Every phase is its own kernel (the kernel boundaries are the barriers).  The
// last CTA of a reducing kernel sums its fixed-order partials once and stores
// the scalars for the next kernel, so no CTA waits on a reduction at its start.
constexpr int kSlotT = kSlotRes + 3;  // t.t of the start pass
constexpr int64_t kFsaiGraphMinRows = 1 << 21;  // auto loop form: graph from here (fp32 inner)
constexpr int kFsaiUnroll = 8;                   // inner iterations per graph of the unrolled form
constexpr int kFsaiOuterKernels = 6;             // kernels of one outer step
// Residency of the graph form's phase kernels: 4 CTAs (32 warps) per SM keeps
// the unrolled diagonal-layout loops within 64 registers without spilling.
constexpr int kFsaiPhaseCtas = 4;

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
  if (g.cta == 0 && threadIdx.x == 0) F.a.gs->xflush = 0;  // gf_xadd has finished
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

template <int W>
__global__ void __launch_bounds__(kBlock, kFsaiPhaseCtas) gf_t(FArgs F) {
  const SolveParams& P = F.a.P;
  Grid g = graph_grid();
  const int64_t n = P.A.n;
  const float* r = F.r[F.a.gs->k & 1];
  Acc<float> a;
  for (int64_t i = g.gtid; i < n; i += g.gstride) {
    const float s = ell_row<W>(F.G, i, n, [&](int j) { return r[j]; });
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
    if (!inner) status = kOk;  // this inner solve has nothing to do; the outer loop goes on
  }
  gs->status = status;
  gs->finished = stop ? 1 : 0;
  if constexpr (COND) {
    cudaGraphSetConditional(F.a.h2, stop ? 0u : 1u);
    cudaGraphSetConditional(F.a.h, inner ? 1u : 0u);
  }
}

// p = G^T t, or p = G^T t + beta0 p when the direction is carried over.
template <int W>
__global__ void __launch_bounds__(kBlock, kFsaiPhaseCtas) gf_p0(FArgs F) {
  const SolveParams& P = F.a.P;
  if (F.a.gs->status != kRunning) return;
  Grid g = graph_grid();
  const int64_t n = P.A.n;
  const float beta0 = (float)F.a.gs->beta0;
  float* p = P.V32.p;
  for (int64_t i = g.gtid; i < n; i += g.gstride) {
    const float s = ell_row<W>(F.GT, i, n, [&](int j) { return F.t[j]; });
    p[i] = beta0 != 0.0f ? fmaf(beta0, p[i], s) : s;
  }
}

// x64 += d when the previous inner solve ended (converged or at maxit; not
// after a breakdown, so x keeps the last good iterate).  First node of an
// outer step; gf_res clears the flag.
__global__ void __launch_bounds__(kBlock) gf_xadd(FArgs F) {
  if (!F.a.gs->xflush) return;
  const SolveParams& P = F.a.P;
  Grid g = graph_grid();
  for (int64_t i = g.gtid; i < P.A.n; i += g.gstride) P.x[i] += (double)F.d[i];
}

// a1: q = A p (fp32 loop matrix, W_A / DIA_A as g_spmv), p.q.  The last CTA
// forms alpha = rho / p.q and the breakdown / non-finite test once.
template <int WA, bool DIAA>
__global__ void __launch_bounds__(kBlock) gf_spmv(FArgs F) {
  const SolveParams& P = F.a.P;
  GState* gs = F.a.gs;
  if (gs->status != kRunning) return;
  Grid g = graph_grid();
  double v[1], pq[1];
  if constexpr (WA > 0) v[0] = spmv_phase_w<float, false, WA, DIAA>(P.S32, P.V32.p, P.V32.q, g);
  else v[0] = spmv_phase<float, false>(P.S32, P.V32.p, P.V32.q, g);
  if (!publish_last<1>(v, P.part + kSlotPQ * (size_t)P.pstride, g, &gs->ctr_q, pq)) return;
  if (threadIdx.x == 0) {
    const double rho = gs->rho;
    const int st = (!isfinite(pq[0]) || !isfinite(rho)) ? kNumeric : (pq[0] <= 0.0 ? kBreakdown : 0);
    gs->alpha = rho / pq[0];
    if (st) gs->status = st;
  }
}

// a2: r' = r - alpha q (into the other r buffer), t = G r' (r' of neighbour
// rows recomputed from r and q), d += alpha p; partials (t.t = r'.z, r'.r').
// The last CTA forms beta, the inner test and the next loop state.
template <int W>
__global__ void __launch_bounds__(kBlock, kFsaiPhaseCtas) gf_upd_r(FArgs F) {
  const SolveParams& P = F.a.P;
  GState* gs = F.a.gs;
  if (gs->status != kRunning) return;
  Grid g = graph_grid();
  const int64_t n = P.A.n;
  const float alpha = (float)gs->alpha;
  const int k = gs->k;
  const float* rc = F.r[k & 1];
  float* rn = F.r[(k + 1) & 1];
  const float* q = P.V32.q;
  const float* p = P.V32.p;
  Acc<float> a_rho, a_rr;
  rows_x2(
      g, n,
      [&](int64_t i) {
        RowUpd<float> u;
        u.r = fmaf(-alpha, q[i], rc[i]);
        u.t = ell_row<W>(F.G, i, n, [&](int j) { return fmaf(-alpha, q[j], rc[j]); });
        u.x = fmaf(alpha, p[i], F.d[i]);
        return u;
      },
      [&](int64_t i, const RowUpd<float>& u) {
        rn[i] = u.r;
        a_rr.add(u.r, u.r);
        F.t[i] = u.t;
        a_rho.add(u.t, u.t);
        F.d[i] = u.x;
      });
  double v[2] = {a_rho.get(), a_rr.get()}, s2[2];
  if (!publish_last<2>(v, P.part + kSlotUpd * (size_t)P.pstride, g, &gs->ctr, s2)) return;
  if (threadIdx.x == 0) {
    const int k1 = k + 1;
    const bool conv = sqrt(s2[1]) <= gs->stop_abs;
    gs->beta = s2[0] / gs->rho;
    gs->rho_k = gs->rho;  // reliable updates: r.z before this step
    gs->rho = s2[0];
    gs->rr = s2[1];
    gs->k = k1;
    if (conv || k1 >= P.maxit) {
      gs->status = conv ? kOk : kNotConverged;
      gs->xflush = 1;
    }
  }
}

// a3: p = G^T t + beta p while the inner solve runs; sets the inner WHILE
// condition (COND) from the state the previous kernels left.
template <int W, bool COND>
__global__ void __launch_bounds__(kBlock, kFsaiPhaseCtas) gf_upd_p(FArgs F) {
  const SolveParams& P = F.a.P;
  const GState* gs = F.a.gs;
  const bool running = gs->status == kRunning;
  if constexpr (COND) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(F.a.h, running ? 1u : 0u);
  }
  if (!running) return;
  Grid g = graph_grid();
  const int64_t n = P.A.n;
  const float beta = (float)gs->beta;
  float* p = P.V32.p;
  rows_x2(
      g, n, [&](int64_t i) { return fmaf(beta, p[i], ell_row<W>(F.GT, i, n, [&](int j) { return F.t[j]; })); },
      [&](int64_t i, float pi) { p[i] = pi; });
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

cg_status build_fsai_graph(cg_handle* h, const FArgs& Fin, int unroll);

// unroll == 0: one launch of the graph with nested WHILE nodes.  unroll > 0:
// the host launches the outer-step graph, then iteration graphs until the
// inner solve leaves kRunning, until the outer loop has finished (every loop
// is bounded by maxit and the outer-step limit, both tested on the device).
cg_status solve_fsai_graph(cg_handle* h, const FArgs& F, bool carry, int unroll, int32_t* iters_out,
                           double* relres_out) {
  FsaiData* f = h->fsai;
  const SolveParams& P = F.a.P;
  if (!f->gexec || f->gkey_b != P.b || f->gkey_x != P.x || f->gkey_tol != P.tol || f->gkey_maxit != P.maxit ||
      f->gkey_tol_in != P.tol_in || f->gkey_outer != P.max_restarts || f->gkey_carry != (int)carry ||
      f->gkey_kind != f->dia || f->gkey_unroll != unroll) {
    const cg_status s = build_fsai_graph(h, F, unroll);
    if (s != CG_OK) return s;
    f->gkey_unroll = unroll;
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
  int64_t launches = 0;
  if (unroll == 0) {
    CGF_CUDA(h, cudaGraphLaunch(f->gexec, h->stream));
  } else {
    auto read_state = [&]() -> cudaError_t {
      cudaError_t e = cudaMemcpyAsync(h->host_gs, h->gs, sizeof(GState), cudaMemcpyDeviceToHost, h->stream);
      return e == cudaSuccess ? cudaStreamSynchronize(h->stream) : e;
    };
    for (;;) {
      CGF_CUDA(h, cudaGraphLaunch(f->gexec, h->stream));
      launches += kFsaiOuterKernels;
      CGF_CUDA(h, read_state());
      if (h->host_gs->finished) break;
      while (h->host_gs->status == kRunning) {
        CGF_CUDA(h, cudaGraphLaunch(f->gexec_it, h->stream));
        launches += 3 * (int64_t)unroll;
        CGF_CUDA(h, read_state());
      }
    }
    CGF_CUDA(h, cudaGraphLaunch(f->gexec_ep, h->stream));
    launches += 1;
  }
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
  h->last.grid_ctas = f->ggrid;
  h->last.relres_true = gs.relres_true;
  h->last.relres_rec = gs.relres_true;
  h->last.kernel_ms = ms;
  h->last.loop_form = unroll > 0 ? 3 : 2;
  if (unroll == 0) launches = kFsaiOuterKernels * (int64_t)(gs.outer + 1) + 3 * (int64_t)gs.k + 1;
  h->last.kernel_launches = (int32_t)std::min<int64_t>(launches, INT32_MAX);
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
  for (cudaGraphExec_t* e : {&f->gexec, &f->gexec_it, &f->gexec_ep}) {
    if (*e) cudaGraphExecDestroy(*e);
    *e = nullptr;
  }
  for (cudaGraph_t* g : {&f->graph, &f->graph_it, &f->graph_ep}) {
    if (*g) cudaGraphDestroy(*g);
    *g = nullptr;
  }
  f->gkey_unroll = -1;
}

// Grids and kernels shared by both graph forms.
struct FsaiGraphPlan {
  FArgs F;
  Csr<double> A;
  const double* x;
  double* q64;
  const void* f_spmv;
  unsigned G, Gq, Gs;
  int w;  // slot form of G and G^T
};

// Slot form of the handle's factor (see kEll / kDiaAny).
int fsai_slots(const FsaiData* f) {
  if (!f->dia) return kEll;
  return (f->nd >= 3 && f->nd <= 5) ? f->nd : kDiaAny;
}

// The instantiation of a kernel template for slot form w.
template <class Pick>
const void* by_slots(int w) {
  switch (w) {
    case 3: return Pick::template fn<3>();
    case 4: return Pick::template fn<4>();
    case 5: return Pick::template fn<5>();
    case kEll: return Pick::template fn<kEll>();
    default: return Pick::template fn<kDiaAny>();
  }
}
struct PickT { template <int W> static const void* fn() { return (const void*)gf_t<W>; } };
struct PickP0 { template <int W> static const void* fn() { return (const void*)gf_p0<W>; } };
struct PickUpdR { template <int W> static const void* fn() { return (const void*)gf_upd_r<W>; } };
// gf_spmv for the loop matrix's uniform slice width uw (as the fp32 g_spmv).
const void* gf_spmv_for(int uw, bool dia) {
  switch (uw) {
    case 4: return dia ? (const void*)gf_spmv<4, true> : (const void*)gf_spmv<4, false>;
    case 6: return dia ? (const void*)gf_spmv<6, true> : (const void*)gf_spmv<6, false>;
    case 8: return dia ? (const void*)gf_spmv<8, true> : (const void*)gf_spmv<8, false>;
    case 26: return dia ? (const void*)gf_spmv<26, true> : (const void*)gf_spmv<0, false>;
    default: return (const void*)gf_spmv<0, false>;
  }
}
template <bool COND>
struct PickUpdP { template <int W> static const void* fn() { return (const void*)gf_upd_p<W, COND>; } };
struct Pick64 { template <int W> static const void* fn() { return (const void*)pcg_fsai64_kernel<W>; } };
template <bool CARRY>
struct PickIr { template <int W> static const void* fn() { return (const void*)pcg_fsai_ir_kernel<W, CARRY>; } };

// CTAs of the vector-phase kernels: one wave at the kernels' own residency,
// bounded by the partial slots.
int fsai_graph_grid(const cg_handle* h) {
  const int w = fsai_slots(h->fsai);
  const void* fns[] = {(const void*)gf_res,          by_slots<PickT>(w),           by_slots<PickP0>(w),
                       by_slots<PickUpdR>(w),        by_slots<PickUpdP<true>>(w),  by_slots<PickUpdP<false>>(w),
                       (const void*)gf_xadd,         (const void*)g_flush_ir};
  int per_sm = 1 << 30;
  for (const void* fn : fns) {
    int k = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, fn, kBlock, 0) != cudaSuccess) return 0;
    per_sm = std::min(per_sm, k);
  }
  return std::max(1, std::min(per_sm * h->sm_count, h->grid_part));
}

cudaError_t plan_fsai_graph(cg_handle* h, const FArgs& Fin, FsaiGraphPlan& pl) {
  pl.F = Fin;
  pl.f_spmv = gf_spmv_for(h->uniform_w, h->dia != 0);
  int per_sm = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.f_spmv, kBlock, 0);
  if (e != cudaSuccess) return e;
  // the phase kernels' own residency (fp32, few registers), not the fp64 loop's
  pl.G = (unsigned)fsai_graph_grid(h);
  if (pl.G == 0) return cudaErrorInvalidValue;
  h->fsai->ggrid = (int)pl.G;
  pl.Gq = (unsigned)std::max(1, std::min(per_sm * h->sm_count, h->grid_part));
  pl.F.a.G_spmv = pl.Gq;
  pl.F.a.G_upd = pl.G;
  pl.A = pl.F.a.P.A;
  pl.x = pl.F.a.P.x;
  pl.q64 = pl.F.a.P.V64.q;
  pl.Gs = (unsigned)std::min<int64_t>(std::max<int32_t>(h->nrb, 1), (int64_t)h->sm_count * 64);
  pl.w = fsai_slots(h->fsai);
  return cudaSuccess;
}

// One outer step: x64 += d, q64 = A x, r = fl32(b - q64), t = G r, the start test, p.
// COND selects the start kernel that sets the WHILE conditions.
template <bool COND>
cudaError_t add_outer_step(cudaGraph_t gr, FsaiGraphPlan& pl, cudaGraphNode_t* last) {
  void* a_spmv[] = {&pl.A, &pl.x, &pl.q64};
  void* a_f[] = {&pl.F};
  const void* fns[kFsaiOuterKernels] = {(const void*)gf_xadd,        (const void*)spmv_kernel<double>,
                                        (const void*)gf_res,         by_slots<PickT>(pl.w),
                                        (const void*)gf_start<COND>, by_slots<PickP0>(pl.w)};
  const unsigned grids[kFsaiOuterKernels] = {pl.G, pl.Gs, pl.G, pl.G, 1, pl.G};
  cudaGraphNode_t prev = nullptr, n;
  for (int k = 0; k < kFsaiOuterKernels; ++k) {
    const unsigned block = fns[k] == (const void*)gf_start<COND> ? 32u : (unsigned)kBlock;
    const cudaError_t e = add_node(gr, &n, prev, fns[k], grids[k], block, k == 1 ? a_spmv : a_f);
    if (e != cudaSuccess) return e;
    prev = n;
  }
  *last = prev;
  return cudaSuccess;
}

// One inner iteration after `prev`: q = A p, p.q | r', t = G r', d | p.
template <bool COND>
cudaError_t add_inner_iteration(cudaGraph_t gr, FsaiGraphPlan& pl, cudaGraphNode_t* prev) {
  void* a_f[] = {&pl.F};
  cudaGraphNode_t b1, b2, b3;
  cudaError_t e = add_node(gr, &b1, *prev, pl.f_spmv, pl.Gq, kBlock, a_f);
  if (e == cudaSuccess) e = add_node(gr, &b2, b1, by_slots<PickUpdR>(pl.w), pl.G, kBlock, a_f);
  if (e == cudaSuccess) e = add_node(gr, &b3, b2, by_slots<PickUpdP<COND>>(pl.w), pl.G, kBlock, a_f);
  *prev = b3;
  return e;
}

// The unrolled form: f->graph = one outer step, f->graph_it = `unroll` inner
// iterations (no conditional nodes, so every kernel node can be profiled),
// f->graph_ep = the b = 0 epilogue.
cg_status build_fsai_unrolled(cg_handle* h, const FArgs& Fin, int unroll) {
  FsaiData* f = h->fsai;
  FsaiGraphPlan pl;
  CGF_CUDA(h, plan_fsai_graph(h, Fin, pl));
  cudaGraphNode_t last = nullptr;
  CGF_CUDA(h, add_outer_step<false>(f->graph, pl, &last));
  CGF_CUDA(h, cudaGraphCreate(&f->graph_it, 0));
  cudaGraphNode_t prev = nullptr;
  for (int u = 0; u < unroll; ++u) CGF_CUDA(h, add_inner_iteration<false>(f->graph_it, pl, &prev));
  CGF_CUDA(h, cudaGraphCreate(&f->graph_ep, 0));
  void* a_ga[] = {&pl.F.a};
  cudaGraphNode_t n;
  CGF_CUDA(h, add_node(f->graph_ep, &n, nullptr, (const void*)g_flush_ir, pl.G, kBlock, a_ga));
  CGF_CUDA(h, cudaGraphInstantiate(&f->gexec, f->graph, 0));
  CGF_CUDA(h, cudaGraphInstantiate(&f->gexec_it, f->graph_it, 0));
  CGF_CUDA(h, cudaGraphInstantiate(&f->gexec_ep, f->graph_ep, 0));
  return CG_OK;
}

cg_status build_fsai_graph(cg_handle* h, const FArgs& Fin, int unroll) {
  FsaiData* f = h->fsai;
  destroy_fsai_graph(f);
  cudaGraph_t g;
  CGF_CUDA(h, cudaGraphCreate(&g, 0));
  f->graph = g;
  if (unroll > 0) return build_fsai_unrolled(h, Fin, unroll);
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
  FsaiGraphPlan pl;
  CGF_CUDA(h, plan_fsai_graph(h, F, pl));
  // kernel arguments are copied into the nodes at creation
  cudaGraphNode_t prev = nullptr, n;
  CGF_CUDA(h, add_outer_step<true>(ob, pl, &prev));
  cudaGraphNodeParams ip{};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = inner_h;
  ip.conditional.type = cudaGraphCondTypeWhile;
  ip.conditional.size = 1;
  CGF_CUDA(h, cudaGraphAddNode(&n, ob, &prev, nullptr, 1, &ip));
  cudaGraph_t ib = ip.conditional.phGraph_out[0];
  cudaGraphNode_t bprev = nullptr;
  CGF_CUDA(h, add_inner_iteration<true>(ib, pl, &bprev));
  void* a_ga[] = {&pl.F.a};
  CGF_CUDA(h, add_node(g, &n, on, (const void*)g_flush_ir, pl.G, kBlock, a_ga));
  CGF_CUDA(h, cudaGraphInstantiate(&f->gexec, g, 0));
  return CG_OK;
}

}  // namespace

void cgi::fsai_free(FsaiData* f) {
  if (!f) return;
  void* dev[] = {f->trp,   f->tci,    f->tsrc,   f->g,      f->gsrc,  f->gcol,  f->gval64, f->gval32,
                 f->gtsrc, f->gtcol,  f->gtval64, f->gtval32, f->r0,   f->r1,    f->t,      f->r0_32,
                 f->r1_32, f->t_32,   f->x_32,   f->offs,   f->work,  f->dout,  f->gpart,  f->mlp_o,
                 f->params32, f->trow, f->rpart, f->tslot, f->a32,    f->d32,   f->rs32,  f->rs64};
  for (void* p : dev)
    if (p) cudaFree(p);
  destroy_fsai_graph(f);
  delete f;
}

namespace {

// ---------------------------------------------------------------- pattern
// Device build of the tril(A) pattern.  Pass 1 (thread per row) validates each
// row as the host build does (strictly increasing columns, a diagonal, at most
// kFsaiMaxRow tril entries; the first failing row in row order is reported:
// key row * 4 + code, atomicMin), and counts the row's tril length, each
// column's tril entries (the widest column is G^T's width) and the distinct
// tril offsets (open-addressing table; more than kFsaiMaxDiag -> ELL).
constexpr int kPatSlots = 32;
constexpr unsigned long long kPatNoErr = ~0ull;
struct PatInfo {
  unsigned long long first_err;
  int gw, gtw, overflow, asym;
  int table[kPatSlots];
};

__global__ void tril_count_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                  int32_t* __restrict__ len, int32_t* __restrict__ cnt, PatInfo* info) {
  int my_gw = 0, my_gtw = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k0 = rowptr[i], k1 = rowptr[i + 1];
    int last = -1, l = 0, code = 0;
    for (int k = k0; k < k1; ++k) {
      const int c = colind[k];
      if (c <= last) {
        code = 1;
        break;
      }
      last = c;
      if (c <= i) ++l;
    }
    if (!code) {
      if (l == 0 || colind[k0 + l - 1] != (int)i) code = 2;
      else if (l > kFsaiMaxRow) code = 3;
    }
    if (code) {
      atomicMin(&info->first_err, (unsigned long long)i * 4ull + (unsigned long long)code);
      len[i] = 0;
      continue;
    }
    len[i] = l;
    my_gw = max(my_gw, l);
    for (int m = 0; m < l; ++m) {
      const int j = colind[k0 + m];
      my_gtw = max(my_gtw, atomicAdd(&cnt[j], 1) + 1);
      const int o = j - (int)i;
      unsigned hs = ((unsigned)o * 2654435761u) >> 27;  // 5 bits
      int t = 0;
      for (; t < kPatSlots; ++t, hs = (hs + 1) & (kPatSlots - 1)) {
        const int v = *((volatile int*)&info->table[hs]);
        if (v == o) break;
        if (v == INT32_MIN) {
          const int old = atomicCAS(&info->table[hs], INT32_MIN, o);
          if (old == INT32_MIN || old == o) break;
        }
      }
      if (t == kPatSlots) info->overflow = 1;
    }
  }
  my_gw = __reduce_max_sync(0xffffffffu, my_gw);
  my_gtw = __reduce_max_sync(0xffffffffu, my_gtw);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&info->gw, my_gw);
    atomicMax(&info->gtw, my_gtw);
  }
}

// Pass 2 (thread per row): tril entries e = trp[i] + m are the row's first
// len entries (columns ascending); their column, source index, row and
// diagonal slot; G's ELL slot map (padding: src -1, own column).
struct PatOffs {
  int nd;
  int off[kFsaiMaxDiag];
};
__global__ void tril_fill_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                 const int32_t* __restrict__ trp, int gw, PatOffs po, int32_t* __restrict__ tci,
                                 int32_t* __restrict__ tsrc, int32_t* __restrict__ trow, int8_t* __restrict__ tslot,
                                 int32_t* __restrict__ gsrc, int32_t* __restrict__ gcol) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int e0 = trp[i], l = trp[i + 1] - e0, k0 = rowptr[i];
    for (int m = 0; m < gw; ++m) {
      const int64_t at = (int64_t)m * n + i;
      if (m < l) {
        const int c = colind[k0 + m];
        tci[e0 + m] = c;
        tsrc[e0 + m] = k0 + m;
        trow[e0 + m] = (int32_t)i;
        if (tslot) {
          int sl = 0;
          while (sl < po.nd - 1 && po.off[sl] != c - (int)i) ++sl;
          tslot[e0 + m] = (int8_t)sl;
        }
        gsrc[at] = e0 + m;
        gcol[at] = c;
      } else {
        gsrc[at] = -1;
        gcol[at] = (int32_t)i;
      }
    }
  }
}

// Pass 3 (thread per column j): with a symmetric structure the tril entries
// of column j are (c, j) for the columns c >= j of row j, ascending; entry
// (c, j) is found in row c's tril part by binary search.  A missing mirror or
// a count that differs from pass 1's sets asym (the host build takes over).
__global__ void gt_fill_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                               const int32_t* __restrict__ trp, const int32_t* __restrict__ cnt, int gtw,
                               int32_t* __restrict__ gtsrc, int32_t* __restrict__ gtcol, PatInfo* info) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    int m = 0;
    bool bad = false;
    for (int k = rowptr[j]; k < rowptr[j + 1] && !bad; ++k) {
      const int c = colind[k];
      if (c < (int)j) continue;
      const int a = rowptr[c], lc = trp[c + 1] - trp[c];
      int lo = 0, hi = lc - 1, p = -1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = colind[a + mid];
        if (v == (int)j) {
          p = mid;
          break;
        }
        if (v < (int)j) lo = mid + 1;
        else hi = mid - 1;
      }
      if (p < 0 || m >= gtw) {
        bad = true;
        break;
      }
      gtsrc[(int64_t)m * n + j] = trp[c] + p;
      gtcol[(int64_t)m * n + j] = c;
      ++m;
    }
    if (bad || m != cnt[j]) {
      info->asym = 1;
      continue;
    }
    for (; m < gtw; ++m) {
      gtsrc[(int64_t)m * n + j] = -1;
      gtcol[(int64_t)m * n + j] = (int32_t)j;
    }
  }
}

std::string pattern_error(int code) {
  switch (code) {
    case 1: return "FSAI needs strictly increasing columns in each row";
    case 2: return "FSAI needs a diagonal entry in every row";
    default: return "FSAI: a row of tril(A) has more than " + std::to_string(kFsaiMaxRow) + " entries";
  }
}

// The device build (passes 1-3; the host scans the row lengths).  Leaves
// *fallback = true, and f untouched, when the structure is not symmetric.
cg_status pattern_device(cg_handle* h, FsaiData* f, bool* fallback) {
  *fallback = false;
  const int64_t n = h->n;
  const unsigned nb = blocks_for(n);
  std::vector<void*> tmp;
  struct Guard {
    std::vector<void*>& v;
    ~Guard() {
      for (void* p : v) cudaFree(p);
    }
  } guard{tmp};
  int32_t *len = nullptr, *cnt = nullptr;
  PatInfo* info = nullptr;
  CGF_CUDA(h, cudaMalloc(&len, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)));
  tmp.push_back(len);
  CGF_CUDA(h, cudaMalloc(&cnt, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)));
  tmp.push_back(cnt);
  CGF_CUDA(h, cudaMalloc(&info, sizeof(PatInfo)));
  tmp.push_back(info);
  PatInfo hi{};
  hi.first_err = kPatNoErr;
  for (int t = 0; t < kPatSlots; ++t) hi.table[t] = INT32_MIN;
  CGF_CUDA(h, cudaMemcpy(info, &hi, sizeof(PatInfo), cudaMemcpyHostToDevice));
  if (n > 0) {
    CGF_CUDA(h, cudaMemset(cnt, 0, sizeof(int32_t) * (size_t)n));
    tril_count_kernel<<<nb, 256>>>(n, h->rowptr, h->colind, len, cnt, info);
    CGF_CUDA(h, cudaGetLastError());
  }
  CGF_CUDA(h, cudaMemcpy(&hi, info, sizeof(PatInfo), cudaMemcpyDeviceToHost));
  if (hi.first_err != kPatNoErr) return ffail(h, CG_ERR_INVALID, pattern_error((int)(hi.first_err & 3ull)));
  if (hi.gtw > kFsaiMaxCol)
    return ffail(h, CG_ERR_INVALID, "FSAI: a column of tril(A) has more than " + std::to_string(kFsaiMaxCol) +
                                        " entries");
  std::vector<int32_t> trp((size_t)n + 1, 0);
  if (n > 0) CGF_CUDA(h, cudaMemcpy(trp.data() + 1, len, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < n; ++i) trp[(size_t)i + 1] += trp[(size_t)i];
  const int64_t nt = trp[(size_t)n];
  std::vector<int32_t> toffs;
  for (int t = 0; t < kPatSlots; ++t)
    if (hi.table[t] != INT32_MIN) toffs.push_back(hi.table[t]);
  std::sort(toffs.begin(), toffs.end());
  const bool dia = !hi.overflow && (int)toffs.size() <= kFsaiMaxDiag;
  PatOffs po{};
  po.nd = dia ? (int)toffs.size() : 0;
  for (int m = 0; m < po.nd; ++m) po.off[m] = toffs[(size_t)m];
  const int gw = hi.gw, gtw = hi.gtw;
  FsaiData d{};  // the arrays, moved into f on success
  auto alloc = [&](int32_t** p, int64_t count) -> cudaError_t {
    const cudaError_t e = cudaMalloc(p, sizeof(int32_t) * (size_t)std::max<int64_t>(count, 1));
    if (e == cudaSuccess) tmp.push_back(*p);
    return e;
  };
  CGF_CUDA(h, alloc(&d.trp, n + 1));
  CGF_CUDA(h, alloc(&d.tci, nt));
  CGF_CUDA(h, alloc(&d.tsrc, nt));
  CGF_CUDA(h, alloc(&d.trow, nt));
  CGF_CUDA(h, alloc(&d.gsrc, (int64_t)gw * n));
  CGF_CUDA(h, alloc(&d.gcol, (int64_t)gw * n));
  CGF_CUDA(h, alloc(&d.gtsrc, (int64_t)gtw * n));
  CGF_CUDA(h, alloc(&d.gtcol, (int64_t)gtw * n));
  if (dia) {
    CGF_CUDA(h, cudaMalloc(&d.tslot, (size_t)std::max<int64_t>(nt, 1)));
    tmp.push_back(d.tslot);
  }
  CGF_CUDA(h, cudaMemcpy(d.trp, trp.data(), sizeof(int32_t) * trp.size(), cudaMemcpyHostToDevice));
  if (n > 0) {
    tril_fill_kernel<<<nb, 256>>>(n, h->rowptr, h->colind, d.trp, gw, po, d.tci, d.tsrc, d.trow, d.tslot, d.gsrc,
                                  d.gcol);
    CGF_CUDA(h, cudaGetLastError());
    gt_fill_kernel<<<nb, 256>>>(n, h->rowptr, h->colind, d.trp, cnt, gtw, d.gtsrc, d.gtcol, info);
    CGF_CUDA(h, cudaGetLastError());
  }
  int asym = 0;
  CGF_CUDA(h, cudaMemcpy(&asym, &info->asym, sizeof(int), cudaMemcpyDeviceToHost));
  if (asym) {
    *fallback = true;  // the guard frees every array
    return CG_OK;
  }
  tmp.resize(3);  // keep len, cnt, info for the guard; the pattern arrays move into f
  f->trp = d.trp;
  f->tci = d.tci;
  f->tsrc = d.tsrc;
  f->trow = d.trow;
  f->gsrc = d.gsrc;
  f->gcol = d.gcol;
  f->gtsrc = d.gtsrc;
  f->gtcol = d.gtcol;
  f->tslot = d.tslot;
  f->ntril = nt;
  f->gw = gw;
  f->gtw = gtw;
  f->dia = dia ? 1 : 0;
  f->nd = po.nd;
  for (int m = 0; m < po.nd; ++m) f->doff[m] = po.off[m];
  return CG_OK;
}

// Host build of the pattern (any CSR structure): the fallback when the
// structure is not symmetric, so that column j of tril(A) is not the upper
// half of row j.
cg_status pattern_host(cg_handle* h, FsaiData* f) {
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
  return CG_OK;
}

// Value arrays of both layouts and the loop's work vectors.
cg_status alloc_loop_arrays(cg_handle* h, FsaiData* f) {
  const int64_t n = h->n, nt = f->ntril;
  const size_t nv = (size_t)std::max<int64_t>(n, 1);
  const int gw = std::max(f->gw, f->nd);  // value arrays serve either layout
  const int gtw = std::max(f->gtw, f->nd);
  CGF_CUDA(h, cudaMalloc(&f->g, sizeof(double) * (size_t)std::max<int64_t>(nt, 1)));
  CGF_CUDA(h, cudaMalloc(&f->gval64, sizeof(double) * (size_t)gw * nv));
  CGF_CUDA(h, cudaMalloc(&f->gval32, sizeof(float) * (size_t)gw * nv));
  CGF_CUDA(h, cudaMalloc(&f->gtval64, sizeof(double) * (size_t)gtw * nv));
  CGF_CUDA(h, cudaMalloc(&f->gtval32, sizeof(float) * (size_t)gtw * nv));
  for (double** v : {&f->r0, &f->r1, &f->t}) CGF_CUDA(h, cudaMalloc(v, sizeof(double) * nv));
  for (float** v : {&f->r0_32, &f->r1_32, &f->t_32, &f->x_32}) CGF_CUDA(h, cudaMalloc(v, sizeof(float) * nv));
  return CG_OK;
}

}  // namespace

// Pattern of G (tril(A)) and of G^T, their ELL slot maps and the loop's
// value and vector arrays, once per handle.  Built on the device; the host
// build covers structures that are not symmetric.
cg_status cgi::fsai_pattern(cg_handle* h) {
  if (h->fsai) return CG_OK;
  if (!h->jacobi_ok) return ffail(h, CG_ERR_INVALID, "FSAI needs a positive diagonal in every row");
  FsaiData* f = new FsaiData();
  bool fallback = false;
  cg_status s = pattern_device(h, f, &fallback);
  if (s == CG_OK && fallback) s = pattern_host(h, f);
  if (s == CG_OK) s = alloc_loop_arrays(h, f);
  if (s != CG_OK) {
    cgi::fsai_free(f);
    return s;
  }
  h->fsai = f;
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
  if (!fp64 && (h->loop_mode >= 2 || (h->loop_mode == 0 && n >= kFsaiGraphMinRows))) {
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
    return solve_fsai_graph(h, FA, carry, h->loop_mode == 3 ? kFsaiUnroll : 0, iters_out, relres_out);
  }
  void* args[] = {&F};
  const void* fn;
  const int sw = fsai_slots(f);
  if (fp64) fn = by_slots<Pick64>(sw);
  else if (carry) fn = by_slots<PickIr<true>>(sw);
  else fn = by_slots<PickIr<false>>(sw);
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
