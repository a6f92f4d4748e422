// The CG loop as a CUDA graph with a device-controlled WHILE node (large
// systems).  Each phase of an iteration is its own high-occupancy kernel; a
// kernel boundary is the grid-wide barrier.  The last CTA of a reducing
// kernel sums the fixed-order per-CTA partials once and stores the scalars
// (alpha after the SpMV, beta and the stopping test after the r update) for
// the next kernel; the last CTA of the x/p pass stores the loop state and sets
// the loop condition.  The host launches one graph per solve and reads one
// status word back.
//
//   prologue : q = A x | r = b - q, r^, p, x^, partials | start (1 CTA)
//   WHILE    : q = A^ p, p.q | alpha, r^ -= alpha q, r.z, r.r | beta, x^/p
//   epilogue : flush x on breakdown | q = A x | ||b - q||^2 | final (1 CTA)
//
// The row work is the same device functions as the persistent launch; the
// two forms sum the CTA partials in different fixed orders, so their iterates
// agree to rounding (each form is deterministic on its own).
#pragma once

#include "cg_kernels.cuh"

namespace cg {

constexpr int kRunning = 100;     // loop state status while iterating
constexpr int kNeedRestart = 101; // recursive residual met tol, true residual did not

// Loop state of a graph solve (device memory, zeroed before the first launch).
struct GState {
  double rho;          // r^.r^ of the current residual
  double rr;           // r.r of the current residual
  double bb;           // b.b
  double stop_abs;     // tol ||b||
  double relres_true;  // ||b - A x|| / ||b|| after the epilogue
  int k;               // SpMVs so far (across restarts)
  int k_start;         // k when this launch's loop started
  int status;          // kRunning, cg status, or kNeedRestart
  int started;         // 0 before the first prologue of a solve
  unsigned ctr;        // arrivals of the current x/p pass (last-CTA election)
  int outer;           // refinement: inner solves started
  double rho_k;        // reliable updates: r.z before the last step of the inner solve
  double beta0;        // reliable updates: carry factor of the next inner solve's p
  int finished;        // refinement: the outer loop has stopped (host test of the unrolled form)
  // scalars formed once by the last CTA of the kernel that reduces them
  double alpha;        // rho / p.q of the current iteration
  double beta;         // rho' / rho
  double rho1, rr1;    // rho' and r.r of the new residual (committed by the x/p pass)
  int want_rr;         // Jacobi: the r update also forms r.D r
  int need_rr;         // Jacobi: g_rr must form the exact r.D r before the test
  int fl;              // the loop ends after this iteration | converged << 1
  int xflush;          // FSAI refinement: the inner solve has ended, x64 += d next
  unsigned ctr_q;      // arrivals of the SpMV launch (last-CTA election)
  unsigned ctr_r;      // arrivals of the r-update launch
  unsigned ctr_rr;     // arrivals of the r.D r launch
};

struct GArgs {
  SolveParams P;
  GState* gs;
  cudaGraphConditionalHandle h;   // the CG loop's WHILE node
  cudaGraphConditionalHandle h2;  // refinement: the outer WHILE node
  unsigned G_spmv;  // CTAs of the SpMV kernel (its p.q partials)
  unsigned G_upd;   // CTAs of the vector kernels (their partials)
};

__device__ __forceinline__ Grid graph_grid() { return Grid(nullptr, 0, 0); }

template <typename T> __device__ __forceinline__ const Sell<T>& sell_of(const SolveParams& P);
template <> __device__ __forceinline__ const Sell<double>& sell_of<double>(const SolveParams& P) { return P.S64; }
template <> __device__ __forceinline__ const Sell<float>& sell_of<float>(const SolveParams& P) { return P.S32; }
template <typename T> __device__ __forceinline__ const LoopVecs<T>& vecs_of(const SolveParams& P);
template <> __device__ __forceinline__ const LoopVecs<double>& vecs_of<double>(const SolveParams& P) { return P.V64; }
template <> __device__ __forceinline__ const LoopVecs<float>& vecs_of<float>(const SolveParams& P) { return P.V32; }

// r = b - q (q = A x from the plain CSR kernel); r^ = D^-1/2 r, p = r^,
// x^ = D^1/2 x; partials (r^.r^, r.r, b.b).
template <bool JAC>
__global__ void __launch_bounds__(kBlock) g_res64(GArgs a) {
  const SolveParams& P = a.P;
  Grid g = graph_grid();
  const LoopVecs<double>& V = P.V64;
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = g.gtid; i < P.A.n; i += g.gstride) {
    const double bi = P.b[i];
    const double ri = bi - V.q[i];
    const double rh = JAC ? ri * __ldg(P.disq + i) : ri;
    V.r[i] = rh;
    V.p[i] = rh;
    V.xh[i] = JAC ? P.x[i] * __ldg(P.dsq + i) : P.x[i];
    v[0] += rh * rh;
    v[1] += ri * ri;
    v[2] += bi * bi;
  }
  publish<3>(v, P.part + kSlotRes * (size_t)P.pstride, g);
}

// One CTA: loop state from the prologue partials; sets the WHILE condition
// (COND; the unrolled form compiles no device-side graph call).
template <bool COND>
__global__ void g_start64(GArgs a) {
  const unsigned G = a.G_upd;
  double s[3];
  grid_sum<3>(a.P.part + kSlotRes * (size_t)a.P.pstride, G, s);
  if (threadIdx.x != 0) return;
  GState* gs = a.gs;
  if (!gs->started) {
    gs->started = 1;
    gs->bb = s[2];
    gs->stop_abs = a.P.tol * sqrt(s[2]);
    gs->k = 0;
  }
  gs->rho = s[0];
  gs->rr = s[1];
  gs->k_start = gs->k;
  int status = kRunning;
  if (gs->bb == 0.0) status = kOk;                          // b = 0: x = 0 (written by g_flush)
  else if (sqrt(s[1]) <= gs->stop_abs) status = kOk;       // a4 before the first SpMV
  else if (gs->k >= a.P.maxit) status = kNotConverged;
  gs->status = status;
  gs->ctr = 0;
  if constexpr (COND) cudaGraphSetConditional(a.h, status == kRunning ? 1u : 0u);
}

// a1: q = A^ p, p.q.  W > 0: the matrix has uniform slices of width W (chosen
// on the host, so each width gets its own register budget).  The last CTA
// forms alpha = rho / p.q, the breakdown / non-finite test and whether the r
// update must form r.D r, once for the next kernels.
template <typename T, bool JAC, int W, bool DIA>
__device__ __forceinline__ void spmv_body(const GArgs& a) {
  const SolveParams& P = a.P;
  GState* gs = a.gs;
  if (gs->status != kRunning) return;
  Grid g = graph_grid();
  const Sell<T>& S = sell_of<T>(P);
  const LoopVecs<T>& V = vecs_of<T>(P);
  double v[1], pq[1];
  if constexpr (W > 0) v[0] = spmv_phase_w<T, JAC, W, DIA>(S, V.p, V.q, g);
  else if constexpr (W < 0) v[0] = spmv_phase_csr<T, JAC>(S, V.p, V.q, g);
  else v[0] = spmv_phase<T, JAC>(S, V.p, V.q, g);
  if (!publish_last<1>(v, P.part + kSlotPQ * (size_t)P.pstride, g, &gs->ctr_q, pq)) return;
  if (threadIdx.x == 0) {
    const double rho = gs->rho;
    const int st = (!isfinite(pq[0]) || !isfinite(rho)) ? kNumeric : (pq[0] <= 0.0 ? kBreakdown : 0);
    gs->alpha = rho / pq[0];
    gs->want_rr = JAC && rr_wanted(S, rho, gs->stop_abs * gs->stop_abs);
    if (st) gs->status = st;
  }
}

template <typename T, bool JAC, int W, bool DIA>
__global__ void __launch_bounds__(kBlock) g_spmv(GArgs a) {
  spmv_body<T, JAC, W, DIA>(a);
}

// Wide uniform slices (W > 16) with a budget of 4 resident CTAs per SM: a
// 26-diagonal row keeps half its loads in flight only with ~64 registers
// (left to itself the compiler chose 48 and the loop waited on memory).
template <typename T, bool JAC, int W, bool DIA>
__global__ void __launch_bounds__(kBlock, 4) g_spmv_wide(GArgs a) {
  spmv_body<T, JAC, W, DIA>(a);
}

// Variable-width slices (sliced ELL, SELL-C-sigma and long rows) with a budget
// of 4 resident CTAs per SM (64 registers): the fp64 form spills below that,
// and the loop unrolls four slice columns (kUnrollG) to keep its gathers in flight.
template <typename T, bool JAC>
__global__ void __launch_bounds__(kBlock, 4) g_spmv_gen(GArgs a) {
  spmv_body<T, JAC, 0, false>(a);
}

// The CSR loop layout (W = -1): only the row-block code is compiled in, so
// the kernel fits 6 resident CTAs per SM (the row gathers wait on memory).
template <typename T, bool JAC>
__global__ void __launch_bounds__(kBlock, 6) g_spmv_csr(GArgs a) {
  spmv_body<T, JAC, -1, false>(a);
}

// The stopping decision for r.r = rr after iteration k1: fl = done | conv << 1.
__device__ __forceinline__ int stop_flags(double rr, double stop_abs, int k1, int maxit) {
  const bool conv = sqrt(rr) <= stop_abs;
  return (conv || k1 >= maxit ? 1 : 0) | (conv ? 2 : 0);
}

// a2: r^ -= alpha q; partials (r^.r^, r.r when wanted).  The last CTA forms
// beta and the test (Jacobi with a varying diagonal: from the bound
// dmin rho <= r.D r <= dmax rho, or it leaves the exact r.D r to g_rr).
template <typename T, bool JAC>
__global__ void __launch_bounds__(kBlock) g_upd_r(GArgs a) {
  const SolveParams& P = a.P;
  GState* gs = a.gs;
  if (gs->status != kRunning) return;
  Grid g = graph_grid();
  const Sell<T>& S = sell_of<T>(P);
  const LoopVecs<T>& V = vecs_of<T>(P);
  const T alpha = (T)gs->alpha;
  const bool want_rr = gs->want_rr != 0;
  double v[2] = {0.0, 0.0}, s2[2];
  update_r_phase<T, JAC>(S, V, alpha, want_rr, v[0], v[1], g);
  if (!publish_last<2>(v, P.part + kSlotUpd * (size_t)P.pstride, g, &gs->ctr_r, s2)) return;
  if (threadIdx.x == 0) {
    const double rho = gs->rho;
    const double stop2 = gs->stop_abs * gs->stop_abs;
    double rr = s2[1];
    const bool need = JAC && !want_rr && rr_bound_test(S, s2[0], stop2, &rr) < 0;
    gs->beta = s2[0] / rho;
    gs->rho1 = s2[0];
    gs->rr1 = rr;
    gs->need_rr = need;
    if (!need) gs->fl = stop_flags(rr, gs->stop_abs, gs->k + 1, P.maxit);
  }
}

// Jacobi with a varying diagonal only: when r.r was skipped and the new rho
// falls into the band where it does not decide the test, compute r.r; the
// last CTA takes the test.
template <typename T>
__global__ void __launch_bounds__(kBlock) g_rr(GArgs a) {
  const SolveParams& P = a.P;
  GState* gs = a.gs;
  if (gs->status != kRunning || !gs->need_rr) return;
  Grid g = graph_grid();
  const Sell<T>& S = sell_of<T>(P);
  double v[1] = {rr_phase<T>(S, vecs_of<T>(P), g)}, rr[1];
  if (!publish_last<1>(v, P.part + kSlotRr * (size_t)P.pstride, g, &gs->ctr_rr, rr)) return;
  if (threadIdx.x == 0) {
    gs->rr1 = rr[0];
    gs->fl = stop_flags(rr[0], gs->stop_abs, gs->k + 1, P.maxit);
  }
}

// a3 + a4: beta, convergence; x^ += alpha p and p = r^ + beta p, or on the
// last iteration out = scale (x^ + alpha p) (OUT_ADD: out += ...).  The last
// CTA to finish stores the loop state and sets the WHILE condition.
template <typename T, bool JAC, bool OUT_ADD, bool COND>
__global__ void __launch_bounds__(kBlock) g_upd_xp(GArgs a) {
  const SolveParams& P = a.P;
  Grid g = graph_grid();
  const Sell<T>& S = sell_of<T>(P);
  const LoopVecs<T>& V = vecs_of<T>(P);
  GState* gs = a.gs;
  if (!COND && gs->status != kRunning) return;  // unrolled form: loop already over
  const bool failed = gs->status != kRunning;  // set by g_spmv (breakdown / numeric)
  double rho1 = 0.0, rr1 = 0.0;
  bool done = true, conv = false;
  const int k1 = gs->k + 1;
  if (!failed) {
    // the scalars the previous kernels' last CTAs formed
    const T alpha = (T)gs->alpha;
    const T beta = (T)gs->beta;
    const int fl = gs->fl;
    rho1 = gs->rho1;
    rr1 = gs->rr1;
    conv = (fl & 2) != 0;
    done = (fl & 1) != 0;
    double* out = P.x;
    if (done) update_xp_phase<T, JAC, true, OUT_ADD>(S, V, alpha, beta, out, g);
    else update_xp_phase<T, JAC, false, OUT_ADD>(S, V, alpha, beta, out, g);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&gs->ctr, 1u) == g.G - 1) {  // every CTA has read the state and finished
      gs->ctr = 0;
      if (!failed) {
        gs->rho = rho1;
        gs->rr = rr1;
        gs->k = k1;
        gs->status = done ? (conv ? kOk : kNotConverged) : kRunning;
      }
      __threadfence();
      if constexpr (COND) cudaGraphSetConditional(a.h, (!failed && !done) ? 1u : 0u);
    }
  }
}

// After the loop: on breakdown / numeric error with iterations done, the
// caller's x gets the last iterate; with b = 0 it gets 0.
template <typename T, bool JAC, bool OUT_ADD>
__global__ void __launch_bounds__(kBlock) g_flush(GArgs a) {
  const SolveParams& P = a.P;
  Grid g = graph_grid();
  const Sell<T>& S = sell_of<T>(P);
  const LoopVecs<T>& V = vecs_of<T>(P);
  const GState* gs = a.gs;
  if (gs->bb == 0.0) {
    for (int64_t i = g.gtid; i < S.n; i += g.gstride) P.x[i] = 0.0;
    return;
  }
  if (!(gs->status == kBreakdown || gs->status == kNumeric) || gs->k == gs->k_start) return;
  for (int64_t i = g.gtid; i < S.n; i += g.gstride) {
    const T xo = JAC ? V.xh[i] * __ldg(S.disq + i) : V.xh[i];
    if (OUT_ADD) P.x[i] += (double)xo;
    else P.x[i] = (double)xo;
  }
}

// Partial ||b - q||^2 with q = A x (true residual, a5).
static __global__ void __launch_bounds__(kBlock) g_true(GArgs a) {
  const SolveParams& P = a.P;
  Grid g = graph_grid();
  double v[1] = {0.0};
  for (int64_t i = g.gtid; i < P.A.n; i += g.gstride) {
    const double ri = P.b[i] - P.V64.q[i];
    v[0] += ri * ri;
  }
  publish<1>(v, P.part + kSlotRes * (size_t)P.pstride, g);
}

// One CTA: the true relative residual and the solve's final status.
static __global__ void g_final64(GArgs a) {
  const unsigned G = a.G_upd;
  double s[1];
  grid_sum<1>(a.P.part + kSlotRes * (size_t)a.P.pstride, G, s);
  if (threadIdx.x != 0) return;
  GState* gs = a.gs;
  if (gs->bb == 0.0) {
    gs->relres_true = 0.0;
    gs->status = kOk;
    return;
  }
  const double rel = sqrt(s[0]) / sqrt(gs->bb);
  gs->relres_true = rel;
  if (!isfinite(rel)) gs->status = kNumeric;
  else if (gs->status == kOk && rel > a.P.tol) gs->status = kNeedRestart;
}

// ---------------------------------------------------------------------------
// fp32-inner / fp64-outer refinement (reading R6) as nested WHILE nodes:
//   outer WHILE { q = A x | r = b - q, r^32, p32, d^ = 0, partials | start (1 CTA) |
//                 inner WHILE { SpMV32 | r update | [r.r] | x/p update, x64 += d } }
// The outer condition starts at 1; the start kernel clears it once the fp64
// residual meets tol (or a limit or an error ends the solve), and sets the
// inner condition for the inner solve it prepares.
// ---------------------------------------------------------------------------

template <bool JAC>
__global__ void __launch_bounds__(kBlock) g_res_ir(GArgs a) {
  const SolveParams& P = a.P;
  Grid g = graph_grid();
  const LoopVecs<float>& V = P.V32;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = g.gtid; i < P.A.n; i += g.gstride) {
    const double bi = P.b[i];
    const double ri = bi - P.V64.q[i];
    const float rh = (float)(JAC ? ri * __ldg(P.disq + i) : ri);
    V.r[i] = rh;
    V.p[i] = rh;
    V.xh[i] = 0.0f;
    const double rh2 = (double)rh * (double)rh;
    v[0] += ri * ri;
    v[1] += bi * bi;
    v[2] += rh2;
    v[3] += JAC ? (double)__ldg(P.S32.dn + i) * rh2 : rh2;
  }
  publish<4>(v, P.part + kSlotRes * (size_t)P.pstride, g);
}

// One CTA: fp64 residual test, limits, and the start state of the next inner solve.
template <bool COND>
__global__ void g_start_ir(GArgs a) {
  double s[4];
  grid_sum<4>(a.P.part + kSlotRes * (size_t)a.P.pstride, a.G_upd, s);
  if (threadIdx.x != 0) return;
  GState* gs = a.gs;
  if (!gs->started) {
    gs->started = 1;
    gs->bb = s[1];
    gs->k = 0;
    gs->outer = 0;
    gs->status = kRunning;
  }
  const double rel = gs->bb > 0.0 ? sqrt(s[0]) / sqrt(gs->bb) : 0.0;
  gs->relres_true = rel;
  gs->rr = s[0];
  bool stop = true;
  int status = gs->status;
  if (status == kBreakdown || status == kNumeric) {
    // the previous inner solve failed; x keeps the last good iterate
  } else if (gs->bb == 0.0) {
    status = kOk;  // x = 0, written after the loop
  } else if (!isfinite(rel)) {
    status = kNumeric;
  } else if (rel <= a.P.tol) {
    status = kOk;
  } else if (gs->outer >= a.P.max_restarts || gs->k >= a.P.maxit) {
    status = kNotConverged;
  } else {
    stop = false;
  }
  bool inner = false;
  if (!stop) {
    gs->rho = s[2];
    gs->stop_abs = a.P.tol_in * sqrt(s[3]);
    gs->k_start = gs->k;
    gs->outer += 1;
    gs->ctr = 0;
    status = kRunning;
    inner = !(sqrt(s[3]) <= gs->stop_abs);  // r32 = 0 only if tol_in >= 1
  }
  gs->status = status;
  if constexpr (COND) {
    cudaGraphSetConditional(a.h2, stop ? 0u : 1u);
    cudaGraphSetConditional(a.h, inner ? 1u : 0u);
  }
}

// After the outer loop: b = 0 gives x = 0.
static __global__ void __launch_bounds__(kBlock) g_flush_ir(GArgs a) {
  if (a.gs->bb != 0.0) return;
  Grid g = graph_grid();
  for (int64_t i = g.gtid; i < a.P.A.n; i += g.gstride) a.P.x[i] = 0.0;
}

}  // namespace cg
