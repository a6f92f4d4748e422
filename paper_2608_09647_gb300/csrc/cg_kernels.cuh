// Kernels of the CG hot path (one GPU, everything resident in HBM):
//   a1  CSR SpMV q = A p fused with the p.q partial sum     (Alg. 1; Sec. 3.3 fused SpMV + dot)
//   a2  alpha, r -= alpha q, r.z and r.r partials, x += alpha p
//                                                          (Alg. 1; Sec. 3.3 fused update + r.r)
//   a3  beta, p = z + beta p                               (Alg. 1)
//   a4  convergence test on the device                     (Alg. 1, relative form)
//   a5  true residual ||b - A x|| / ||b|| in fp64         (Sec. 3.1, recomputed residual)
//
// The loop runs as one persistent cooperative launch.  Phases are separated by
// bounded grid barriers; every CTA forms the scalars redundantly from
// fixed-order sums of per-CTA partials, so there is no host round trip per
// iteration and reruns give identical results.
//
// GB300 design of one iteration:
//  * Jacobi is applied as the symmetric scaling A^ = D^-1/2 A D^-1/2, which
//    is algebraically the same iteration (x = D^-1/2 x^, r = D^1/2 r^,
//    r.z = r^.r^, r.r = r^.D r^) and leaves A^ with a unit diagonal, so the
//    loop streams no D^-1 vector and stores no diagonal entries.
//  * Three streaming phases: [q = A^ p, p.q] | [r^ -= alpha q, r.z, r.r] |
//    [x^ += alpha p, p = r^ + beta p]; the x update rides in the p pass, and
//    on the last iteration that pass writes the caller's x directly.
//    (Forming p on the fly inside the SpMV saves one pass and one barrier
//    but doubles the gathered vectors; measured on GB300 that halves the
//    SpMV's bandwidth, so the p update stays a pass of its own.)
//  * The loop matrix is stored as SELL-32 (sliced ELLPACK, slice height 32 =
//    one warp): the off-diagonal entries of 32 consecutive rows are laid out
//    column-major per slice, so lane l of a warp owns row 32 s + l, every
//    matrix load and most gathers are coalesced, the row sum stays in one
//    register, and warps run with no shared memory and no CTA barrier.  The
//    matrix is streamed with evict-first loads so the L2 keeps the vectors
//    that the gathers reuse.  Rows longer than kLongRow entries leave the
//    slices and are summed by a warp each from a compact CSR.
#pragma once

#include "cg_csr.cuh"

namespace cg {

constexpr int kLongRow = 128;              // off-diagonal entries above which a row leaves SELL
constexpr int kUnroll = 8;                 // slice columns whose loads are issued together
constexpr int kUnrollG = 4;                // the same in the generic (variable-width) slice loop
constexpr double kIrTolInner = 1e-4;       // default inner tolerance: refinement (restarting)
constexpr double kRuTolInner = 1e-1;       // default update threshold: reliable updates
constexpr int kMaxDiag = 32;               // most distinct offsets of the diagonal (DIA) layout
constexpr int kSellSigma = 256;            // rows sorted by length within windows of this many
constexpr double kCsrPadLimit = 1.3;       // slices padding the entries by more: the CSR loop layout

// --------------------------------------------------------------------------
// Persistent solver launch
// --------------------------------------------------------------------------

// Off-diagonal part of the loop matrix (A^ with Jacobi, A without) in
// SELL-32 form, or in its sliced-diagonal special case (dia != 0): when every
// off-diagonal entry lies on one of ndiag <= kMaxDiag diagonals j - i = delta[m]
// and few slots are empty, slice column m holds diagonal m, the column index
// of row i is i + delta[m] (clamped into range for the zero-valued slots) and
// no column array is stored.  Otherwise:  Slice s holds rows [32 s, 32 s + 32); its entries occupy
// [soff[s], soff[s+1]) in units of 32 (column m of the slice is the 32
// consecutive elements at (soff[s] + m) * 32; lane l = row 32 s + l).  Short
// rows are padded to the slice width with (column = own row, value = 0).
// Rows with more than kLongRow off-diagonal entries are marked in lmask and
// kept in a compact CSR (lrow / lptr / lcol / lval) instead.
template <typename T>
struct Sell {
  int64_t n;
  int32_t nslices;
  int32_t uw;  // >= 0: every slice has width uw and no row is long (soff, lmask unread)
  int32_t dia;                // 1: sliced-diagonal layout, width uw = number of diagonals
  int32_t delta[kMaxDiag];    // diagonal offsets (dia only)
  const int32_t* __restrict__ soff;
  const uint32_t* __restrict__ lmask;
  const int32_t* __restrict__ col;
  const T* __restrict__ val;
  int32_t nlong;
  const int32_t* __restrict__ lrow;
  const int32_t* __restrict__ lptr;
  const int32_t* __restrict__ lcol;
  const T* __restrict__ lval;
  const int32_t* __restrict__ perm;  // row at each slice position (SELL-C-sigma; n = none), or null
  int32_t csr;                 // 1: the loop matrix is a CSR of the off-diagonal entries (col / val),
  int32_t nrb;                 //    cut into nrb row blocks rb[] over the row pointers rptr[]
  const int32_t* __restrict__ rptr;
  const int32_t* __restrict__ rb;
  const T* __restrict__ dg;    // diagonal of the loop matrix (unused with Jacobi: unit diagonal)
  const T* __restrict__ dn;    // A_ii weights of the true residual norm (Jacobi)
  const T* __restrict__ disq;  // 1/sqrt(A_ii) mapping x^ back to x (Jacobi)
  double dmin, dmax;           // range of A_ii (Jacobi): dmin r^.r^ <= r.r <= dmax r^.r^
};

// With Jacobi the stopping test needs r.r = r^.D r^, two more fp64 operations
// and one more vector per row.  Since dmin rho <= r.r <= dmax rho, the test is
// decided by rho alone except in the band stop^2 / dmax < rho <= stop^2 / dmin
// (empty when the diagonal is constant).  The r update computes r.r only once
// dmin rho comes within kRrMargin of stop^2; if rho jumps into the band before
// that, one extra pass computes r.r, so the test stays exact.
constexpr double kRrMargin = 64.0;

template <typename T>
__device__ __forceinline__ bool rr_wanted(const Sell<T>& S, double rho, double stop2) {
  return S.dmin != S.dmax && S.dmin * rho <= kRrMargin * stop2;
}

// Decide sqrt(r.r) <= stop from rho: 1 converged, 0 not converged, -1 unknown.
// *rr gets dmax rho (exact for a constant diagonal).
template <typename T>
__device__ __forceinline__ int rr_bound_test(const Sell<T>& S, double rho, double stop2, double* rr) {
  *rr = S.dmax * rho;
  if (S.dmax * rho <= stop2) return 1;
  if (S.dmin * rho > stop2) return 0;
  return -1;
}

// Work vectors of the loop on type T.
template <typename T>
struct LoopVecs {
  T* r;       // r^ (scaled residual)
  T* p;       // search direction
  T* q;       // A^ p
  T* xh;      // x^ (scaled iterate; the inner correction d^ when refining)
};

struct SolveParams {
  Csr<double> A;          // caller's fp64 matrix (true residual)
  Sell<double> S64;       // fp64 loop matrix
  Sell<float> S32;        // fp32 loop matrix (refinement)
  LoopVecs<double> V64;
  LoopVecs<float> V32;
  const double* b;
  double* x;
  const double* dsq;      // sqrt(A_ii) (Jacobi)
  const double* disq;     // 1/sqrt(A_ii) (Jacobi)
  double* part;           // per-CTA partials: kParts slots of pstride doubles
  int pstride;            // slot stride (>= the grid of every loop kernel)
  DevState* st;
  double tol;             // outer relative tolerance
  double tol_in;          // inner tolerance (refinement)
  int maxit;              // SpMV cap (total inner iterations when refining)
  int max_restarts;       // residual replacements (fp64) / refinement steps
  uint64_t timeout_ns;
  unsigned skip_seq;
  int timers;             // accumulate CTA 0 phase times into st->tphase
};

// Partial-sum slots (each G doubles): 0 = p.q, 1 = r.r fallback, 2/3 = the
// update phase, 4..7 = the residual phase.  Disjoint slots mean a CTA never overwrites a
// partial that a slower CTA still has to read.
constexpr int kParts = 8;
constexpr int kSlotPQ = 0, kSlotRr = 1, kSlotUpd = 2, kSlotRes = 4;

// Grid coordinates and the barrier sequence of one persistent launch.
struct Grid {
  unsigned G, cta;
  int64_t gtid, gstride;
  DevState* st;
  uint64_t timeout_ns;
  unsigned seq, skip_seq;
  __device__ Grid(DevState* s, uint64_t to, unsigned skip)
      : G(gridDim.x), cta(blockIdx.x), gtid((int64_t)blockIdx.x * kBlock + threadIdx.x),
        gstride((int64_t)gridDim.x * kBlock), st(s), timeout_ns(to), seq(0), skip_seq(skip) {}
  __device__ __forceinline__ bool sync() { return grid_barrier(st, G, timeout_ns, ++seq, skip_seq); }
};

// Write this CTA's block sums of v[0..NV) into part[j*G + cta] (v is
// consumed: afterwards it holds the sums in thread 0 only).
template <int NV, bool EXACT = true>
__device__ __forceinline__ void publish(double (&v)[NV], double* part, const Grid& g) {
  cta_sum0<NV, EXACT>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) part[(size_t)j * g.G + g.cta] = v[j];
  }
}

// publish, then elect the last CTA of the launch to arrive (counter *ctr):
// it sums the G partials once (thread t takes partials t, t + kBlock, ...;
// then cta_sum0), leaves the totals in thread 0's tot, resets the counter and
// returns true in every one of its threads.  Consumers then read finished
// scalars instead of re-summing G partials in every CTA.  Writer: partial,
// fence, counter; reader: counter, fence, L2 loads (no stale L1 lines).
template <int NV>
__device__ __forceinline__ bool publish_last(double (&v)[NV], double* part, const Grid& g, unsigned* ctr,
                                             double (&tot)[NV]) {
  __shared__ int s_last;
  publish<NV>(v, part, g);
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(ctr, 1u) == g.G - 1;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double t = 0.0;
    for (unsigned c = threadIdx.x; c < g.G; c += kBlock) t += __ldcg(part + (size_t)j * g.G + c);
    tot[j] = t;
  }
  cta_sum0<NV>(tot);
  if (threadIdx.x == 0) *ctr = 0;
  return true;
}

template <typename T> struct Vec;
template <> struct Vec<double> { using type = double2; static constexpr int N = 2; };
template <> struct Vec<float> { using type = float4; static constexpr int N = 4; };

template <typename T, typename VT>
__device__ __forceinline__ T& lane(VT& v, int j) {
  return reinterpret_cast<T*>(&v)[j];
}
template <typename T, typename VT>
__device__ __forceinline__ T lane_c(const VT& v, int j) {
  return reinterpret_cast<const T*>(&v)[j];
}

// Per-thread dot-product accumulator.  fp64: fused multiply-add.  fp32 (the
// refinement's inner solve): fp32 products summed with Kahan compensation, so
// the per-thread partial is accurate to about one fp32 rounding without any
// fp64 instruction (GB300 issues 64 fp32 FMAs per fp64 FMA); partials are
// combined in fp64 across threads and CTAs.
template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float y = __fmul_rn(a, b) - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Status codes shared with the host API (values of cg_status).
constexpr int kOk = 0, kNotConverged = 1, kBreakdown = -2, kNumeric = -3, kTimeout = -4;

// CTA-local phase timer (CTA 0, thread 0, when enabled).
struct PhaseClock {
  bool on;
  uint64_t t;
  __device__ PhaseClock(bool enabled) : on(enabled && blockIdx.x == 0 && threadIdx.x == 0), t(0) {
    if (on) t = global_timer_ns();
  }
  __device__ __forceinline__ void lap(DevState* st, int slot) {
    if (on) {
      const uint64_t now = global_timer_ns();
      st->tphase[slot] += now - t;
      t = now;
    }
  }
};

// Streaming (evict-first) loads for the matrix, read once per iteration.
__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }

// a1 over the grid for uniform slices of compile-time width W (no long rows):
// every load of a slice is issued at once and the register footprint is
// exactly what W needs, which keeps occupancy high.  DIA: the column of slot m
// is computed from delta[m] instead of loaded.  The diagonal term starts the
// fused multiply-add chain, so each row costs W + 1 fp64 FMAs with the p.q term.
// One slice's off-diagonal sum for uniform width W: loads of a chunk of CH
// columns are issued together, then the multiply-adds.  DIA: the column of
// slot m is i + delta[m], clamped into [0, n) with two 32-bit min/max (only
// zero-valued slots of the first and last slices ever need the clamp).
template <typename T, int W, bool DIA>
__device__ __forceinline__ T slice_sum(const Sell<T>& S, const T* __restrict__ p, int64_t s,
                                       int i32, int lane, T acc) {
  constexpr int CH = W > 16 ? (W + 1) / 2 : W;
  const T* vp = S.val + s * (W * 32) + lane;
  const int nm1 = (int)S.n - 1;
#pragma unroll
  for (int m0 = 0; m0 < W; m0 += CH) {
    T v[CH], pc[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int m = m0 + u;
      if (m < W) {
        v[u] = ld_stream(vp + m * 32);
        const int c = DIA ? min(max(i32 + S.delta[m], 0), nm1)
                          : ld_stream(S.col + s * (W * 32) + lane + m * 32);
        pc[u] = p[c];
      }
    }
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (m0 + u < W) acc = fma(v[u], pc[u], acc);
  }
  return acc;
}

// a1 over the grid for uniform slices of compile-time width W (no long rows).
// Warps take slices round-robin, so at any moment the grid works on one
// contiguous band of rows and the neighbours' lines are shared through L2.
// The diagonal term starts the fused multiply-add chain: W + 1 FMAs per row
// with the p.q term.
template <typename T, bool JAC, int W, bool DIA>
__device__ __forceinline__ double spmv_phase_w(const Sell<T>& S, const T* __restrict__ p,
                                               T* __restrict__ q, const Grid& g) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)g.cta * kWarps + (int)(threadIdx.x >> 5);
  const int Wt = (int)g.G * kWarps;
  const int n = (int)S.n;
  Acc<T> dot;
  int s = gw;
  if constexpr (sizeof(T) == 4 && W <= 8) {
    // fp32 loops at 2 CTAs per SM: a warp's slices cost one L2 round trip each, so
    // two slices go together, every load of both issued before the first product
    // (the same arithmetic and order as one slice at a time)
    const int nm1 = n - 1;
    for (; s + Wt < S.nslices; s += 2 * Wt) {
      T v[2][W], pc[2][W], pi[2], acc[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int sh = s + h * Wt, i = sh * 32 + lane;
        const bool live = i < n;
        pi[h] = T(0);
        T dgi = T(1);
        if (live) {
          pi[h] = p[i];
          if (!JAC) dgi = __ldg(S.dg + i);
        }
        acc[h] = JAC ? pi[h] : dgi * pi[h];
        const T* vp = S.val + (int64_t)sh * (W * 32) + lane;
#pragma unroll
        for (int m = 0; m < W; ++m) {
          v[h][m] = ld_stream(vp + m * 32);
          const int c = DIA ? min(max(i + S.delta[m], 0), nm1) : ld_stream(S.col + (int64_t)sh * (W * 32) + lane + m * 32);
          pc[h][m] = p[c];
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int m = 0; m < W; ++m) acc[h] = fma(v[h][m], pc[h][m], acc[h]);
        const int i = (s + h * Wt) * 32 + lane;
        if (i < n) {
          q[i] = acc[h];
          dot.add(pi[h], acc[h]);
        }
      }
    }
  }
  for (; s < S.nslices; s += Wt) {
    const int i = s * 32 + lane;
    const bool live = i < n;
    T pi = T(0), dgi = T(1);
    if (live) {
      pi = p[i];
      if (!JAC) dgi = __ldg(S.dg + i);
    }
    T acc = JAC ? pi : dgi * pi;
    acc = slice_sum<T, W, DIA>(S, p, s, i, lane, acc);
    if (live) {
      q[i] = acc;
      dot.add(pi, acc);
    }
  }
  return dot.get();
}

// Sliced-diagonal layout of any width up to kMaxDiag (loads in groups of kUnroll).
template <typename T, bool JAC>
__device__ __forceinline__ double spmv_phase_dia(const Sell<T>& S, const T* __restrict__ p,
                                                 T* __restrict__ q, const Grid& g) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)g.cta * kWarps + (int)(threadIdx.x >> 5);
  const int Wt = (int)g.G * kWarps;
  const int64_t n = S.n;
  const int w = S.uw;
  Acc<T> dot;
  for (int s = gw; s < S.nslices; s += Wt) {
    const int64_t i = (int64_t)s * 32 + lane;
    const bool live = i < n;
    T pi = T(0), dgi = T(1);
    if (live) {
      pi = p[i];
      if (!JAC) dgi = __ldg(S.dg + i);
    }
    const T* vp = S.val + (int64_t)s * w * 32 + lane;
    const int64_t r0 = (int64_t)s * 32;
    const bool inner = r0 + S.delta[0] >= 0 && r0 + 31 + S.delta[w - 1] < n;
    const T* pb = p + i;
    T acc = JAC ? pi : dgi * pi;
    for (int m0 = 0; m0 < w; m0 += kUnroll) {
      T v[kUnroll], pc[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (m0 + u < w) {
          v[u] = ld_stream(vp + (m0 + u) * 32);
          if (inner) {
            pc[u] = pb[S.delta[m0 + u]];
          } else {
            const int64_t cc = i + S.delta[m0 + u];
            pc[u] = p[cc < 0 ? 0 : (cc >= n ? n - 1 : cc)];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (m0 + u < w) acc = fma(v[u], pc[u], acc);
    }
    if (live) {
      q[i] = acc;
      dot.add(pi, acc);
    }
  }
  return dot.get();
}

// The CSR loop layout (matrices whose rows are too uneven for slices): one row
// block of q = A^ p, staged as the caller-CSR SpMV stages it (16-byte loads of
// columns and values into shared memory), rows of at most kThreadRow entries by
// a thread, longer ones by a warp, a row beyond the block cap by the CTA; the
// diagonal term starts each row's sum; the row's p_i q_i goes to dot.
template <typename T> struct Quad;
template <> struct Quad<double> {
  __device__ static void load(const double* v, double (&o)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(v));
    const double2 b = __ldg(reinterpret_cast<const double2*>(v + 2));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  __device__ static void store(double* s, const double (&o)[4]) {
    reinterpret_cast<double2*>(s)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2*>(s)[1] = make_double2(o[2], o[3]);
  }
};
template <> struct Quad<float> {
  __device__ static void load(const float* v, float (&o)[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(v));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  }
  __device__ static void store(float* s, const float (&o)[4]) {
    reinterpret_cast<float4*>(s)[0] = make_float4(o[0], o[1], o[2], o[3]);
  }
};

constexpr int kRowStep = 4;  // a row's gathers in flight together in the CSR loop layout

template <typename T, bool JAC>
__device__ __forceinline__ void loop_rowblock(const Sell<T>& S, const T* __restrict__ p, T* __restrict__ q, int b,
                                              int* s_col, T* s_val, int* s_med, int* s_nmed, Acc<T>& dot) {
  // positions [r0, r1) of block b; position ps holds row S.perm[ps] (the rows of a
  // block sorted by descending length) with entries at [rptr[ps], rptr[ps+1])
  const int r0 = __ldg(S.rb + b), r1 = __ldg(S.rb + b + 1);
  const int k0 = __ldg(S.rptr + r0), k1 = __ldg(S.rptr + r1);
  const int t = threadIdx.x;
  if (k1 - k0 > kCapV) {  // one long row: strided FMA, fixed tree
    double acc = 0.0;
    for (int k = k0 + t; k < k1; k += kBlock) acc = fma((double)__ldg(S.val + k), (double)p[__ldg(S.col + k)], acc);
    double v[1] = {acc};
    block_sum<1>(v);
    if (t == 0) {
      const int i = __ldg(S.perm + r0);
      const T pi = p[i];
      const T qi = (JAC ? pi : __ldg(S.dg + i) * pi) + (T)v[0];
      q[i] = qi;
      dot.add(pi, qi);
    }
    return;
  }
  const int a0 = k0 & ~3;  // the loop arrays start on 256-byte boundaries
  const int nq = (k1 - a0 + 3) >> 2;
  if (t == 0) *s_nmed = 0;
#pragma unroll
  for (int j = 0; j < kQuadPasses; ++j) {
    const int qd = t + j * kBlock;
    if (qd >= nq) continue;
    const int k = a0 + 4 * qd;
    int c[4] = {0, 0, 0, 0};
    T v[4] = {T(0), T(0), T(0), T(0)};
    if (k + 4 <= k1) {
      const int4 c4 = __ldg(reinterpret_cast<const int4*>(S.col + k));
      c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
      Quad<T>::load(S.val + k, v);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u < k1) {
          c[u] = __ldg(S.col + k + u);
          v[u] = __ldg(S.val + k + u);
        }
    }
    *reinterpret_cast<int4*>(s_col + 4 * qd) = make_int4(c[0], c[1], c[2], c[3]);
    Quad<T>::store(s_val + 4 * qd, v);
  }
  __syncthreads();
  const int ps = r0 + t;
  int a = 0, len = 0, i = 0;
  if (ps < r1) {
    a = __ldg(S.rptr + ps) - a0;
    len = __ldg(S.rptr + ps + 1) - a0 - a;
    i = __ldg(S.perm + ps);
  }
  // (the rows of a block are sorted by length, so the first warps hold the long
  // ones: those are shared out among all warps instead of kept by one)
  if (len > kThreadRow) {
    s_med[atomicAdd(s_nmed, 1)] = ps;
    len = -1;
  }
  // a warp's rows, one a thread: the FMA chain runs to the warp's longest row
  // (one fp64 warp instruction per step), each lane keeping its sum past its
  // own row's end
  const int wlen = __reduce_max_sync(0xffffffffu, len);
  if (len >= 0 && ps < r1) {
    const T pi = p[i];
    T acc = JAC ? pi : __ldg(S.dg + i) * pi;
    int k = 0;
    for (; k + kRowStep <= wlen; k += kRowStep) {  // kRowStep gathers in flight together
      T xv[kRowStep], vv[kRowStep];
#pragma unroll
      for (int u = 0; u < kRowStep; ++u) {
        const bool in = k + u < len;
        vv[u] = in ? s_val[a + k + u] : T(0);
        xv[u] = in ? p[s_col[a + k + u]] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kRowStep; ++u) {
        const T nx = fma(vv[u], xv[u], acc);
        acc = k + u < len ? nx : acc;
      }
    }
    for (; k < wlen; ++k) {  // the warp's last steps, one at a time
      const bool in = k < len;
      const T nx = fma(in ? s_val[a + k] : T(0), in ? p[s_col[a + k]] : T(0), acc);
      acc = in ? nx : acc;
    }
    q[i] = acc;
    dot.add(pi, acc);
  }
  __syncthreads();
  const int nmed = *s_nmed;
  const int lane = t & 31;
  for (int m = t >> 5; m < nmed; m += kWarps) {
    const int pm = s_med[m];
    const int row = __ldg(S.perm + pm);
    const int am = __ldg(S.rptr + pm) - a0, em = __ldg(S.rptr + pm + 1) - a0;
    T acc = T(0);
    for (int k = am + lane; k < em; k += 32) acc = fma(s_val[k], p[s_col[k]], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const T pi = p[row];
      const T qi = (JAC ? pi : __ldg(S.dg + row) * pi) + acc;
      q[row] = qi;
      dot.add(pi, qi);
    }
  }
  __syncthreads();  // the staging buffers are reused by the next row block
}

template <typename T, bool JAC>
__device__ __forceinline__ double spmv_phase_csr(const Sell<T>& S, const T* __restrict__ p, T* __restrict__ q,
                                                 const Grid& g) {
  __shared__ __align__(16) int s_col[kCap];
  __shared__ __align__(16) T s_val[kCap];
  __shared__ int s_med[kBlock];
  __shared__ int s_nmed;
  Acc<T> dot;
  for (int b = (int)g.cta; b < S.nrb; b += (int)g.G) loop_rowblock<T, JAC>(S, p, q, b, s_col, s_val, s_med, &s_nmed, dot);
  return dot.get();
}

// a1 over the grid: q = A^ p and this thread's share of p.q.  Warps take
// slices round-robin; long rows are summed by a warp each.  Uniform slices of
// width 4, 6 or 8 go to the specialised loop.
template <typename T, bool JAC>
__device__ __forceinline__ double spmv_phase(const Sell<T>& S, const T* __restrict__ p,
                                             T* __restrict__ q, const Grid& g) {
  if (S.csr) return spmv_phase_csr<T, JAC>(S, p, q, g);
  if (S.dia) {
    if (S.uw == 4) return spmv_phase_w<T, JAC, 4, true>(S, p, q, g);
    if (S.uw == 6) return spmv_phase_w<T, JAC, 6, true>(S, p, q, g);
    if (S.uw == 8) return spmv_phase_w<T, JAC, 8, true>(S, p, q, g);
    if (S.uw == 26) return spmv_phase_w<T, JAC, 26, true>(S, p, q, g);
    return spmv_phase_dia<T, JAC>(S, p, q, g);
  }
  if (S.uw == 4) return spmv_phase_w<T, JAC, 4, false>(S, p, q, g);
  if (S.uw == 6) return spmv_phase_w<T, JAC, 6, false>(S, p, q, g);
  if (S.uw == 8) return spmv_phase_w<T, JAC, 8, false>(S, p, q, g);
  const int lane = threadIdx.x & 31;
  const int gw = (int)g.cta * kWarps + (int)(threadIdx.x >> 5);
  const int W = (int)g.G * kWarps;
  const int64_t n = S.n;
  Acc<T> dot;
  for (int s = gw; s < S.nslices; s += W) {
    // slice position -> row: with SELL-C-sigma the rows of a window are sorted
    // by length, so one slice holds rows of similar length (little padding)
    const int64_t pos = (int64_t)s * 32 + lane;
    const int64_t i = S.perm ? (int64_t)__ldg(S.perm + pos) : pos;
    int o0, w;
    uint32_t lm;
    if (S.uw >= 0) {  // uniform slices: offsets are arithmetic, no metadata loads
      o0 = s * S.uw;
      w = S.uw;
      lm = 0u;
    } else {
      o0 = __ldg(S.soff + s);
      w = __ldg(S.soff + s + 1) - o0;
      lm = __ldg(S.lmask + s);
    }
    T pi = T(0), dgi = T(1);
    if (i < n) {
      pi = p[i];
      if (!JAC) dgi = __ldg(S.dg + i);
    }
    const int32_t* cp = S.col + (int64_t)o0 * 32 + lane;
    const T* vp = S.val + (int64_t)o0 * 32 + lane;
    T acc = JAC ? pi : dgi * pi;
    for (int m0 = 0; m0 < w; m0 += kUnrollG) {
      int c[kUnrollG];
      T v[kUnrollG], pc[kUnrollG];
#pragma unroll
      for (int u = 0; u < kUnrollG; ++u) {
        if (m0 + u < w) {
          c[u] = ld_stream(cp + (m0 + u) * 32);
          v[u] = ld_stream(vp + (m0 + u) * 32);
        }
      }
#pragma unroll
      for (int u = 0; u < kUnrollG; ++u)
        if (m0 + u < w) pc[u] = p[c[u]];
#pragma unroll
      for (int u = 0; u < kUnrollG; ++u)
        if (m0 + u < w) acc = fma(v[u], pc[u], acc);
    }
    if (i < n && !((lm >> lane) & 1u)) {
      q[i] = acc;
      dot.add(pi, acc);
    }
  }
  // long rows: one warp per row, lanes stride, fixed xor tree
  for (int l = gw; l < S.nlong; l += W) {
    const int i = __ldg(S.lrow + l);
    const int a = __ldg(S.lptr + l), e = __ldg(S.lptr + l + 1);
    T acc = T(0);
    for (int k = a + lane; k < e; k += 32) acc = fma(__ldg(S.lval + k), p[__ldg(S.lcol + k)], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const T pi = p[i];
      const T qi = (JAC ? pi : __ldg(S.dg + i) * pi) + acc;
      q[i] = qi;
      dot.add(pi, qi);
    }
  }
  return dot.get();
}

// a2 over the grid: r^ -= alpha q; rho = r^.r^ (= r.z); rr = r^.D r^ (= r.r,
// Jacobi) or rho.  Two 16-byte vectors per thread per trip, loads first.
template <typename T, bool JAC>
__device__ __forceinline__ void update_r_phase(const Sell<T>& S, const LoopVecs<T>& V, T alpha,
                                               bool want_rr, double& rho, double& rr,
                                               const Grid& g) {
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::N;
  const int64_t n = S.n;
  const int64_t nv = n / VN;
  VT* r = reinterpret_cast<VT*>(V.r);
  const VT* q = reinterpret_cast<const VT*>(V.q);
  const VT* dn = reinterpret_cast<const VT*>(S.dn);
  const bool with_rr = JAC && want_rr;
  Acc<T> a_rho, a_rr;
  for (int64_t i0 = g.gtid; i0 < nv; i0 += 2 * g.gstride) {
    const int64_t i1 = i0 + g.gstride;
    const bool two = i1 < nv;
    VT rv[2], qv[2], dv[2];
    rv[0] = r[i0];
    qv[0] = q[i0];
    if (with_rr) dv[0] = __ldg(dn + i0);
    if (two) {
      rv[1] = r[i1];
      qv[1] = q[i1];
      if (with_rr) dv[1] = __ldg(dn + i1);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !two) break;
#pragma unroll
      for (int j = 0; j < VN; ++j) {
        const T ri = fma(-alpha, lane_c<T>(qv[h], j), lane<T>(rv[h], j));
        lane<T>(rv[h], j) = ri;
        a_rho.add(ri, ri);
        if (with_rr) a_rr.add(lane<T>(dv[h], j) * ri, ri);
      }
    }
    r[i0] = rv[0];
    if (two) r[i1] = rv[1];
  }
  for (int64_t i = nv * VN + g.gtid; i < n; i += g.gstride) {
    const T ri = fma(-alpha, V.q[i], V.r[i]);
    V.r[i] = ri;
    a_rho.add(ri, ri);
    if (with_rr) a_rr.add(__ldg(S.dn + i) * ri, ri);
  }
  rho += a_rho.get();
  rr += a_rr.get();
  if (!JAC) rr = rho;
}

// r.r = r^.D r^ from the current r^ (the exact-test fallback).
template <typename T>
__device__ __forceinline__ double rr_phase(const Sell<T>& S, const LoopVecs<T>& V, const Grid& g) {
  Acc<T> rr;
  for (int64_t i = g.gtid; i < S.n; i += g.gstride) {
    const T ri = V.r[i];
    rr.add(__ldg(S.dn + i) * ri, ri);
  }
  return rr.get();
}

// a3 over the grid: x^ += alpha p; p = r^ + beta p.  On the last iteration
// (FINAL) the p update is skipped and the caller's x is written instead:
// out = scale (x^ + alpha p), or out += fl64(scale (x^ + alpha p)) (OUT_ADD).
template <typename T, bool JAC, bool FINAL, bool OUT_ADD>
__device__ __forceinline__ void update_xp_phase(const Sell<T>& S, const LoopVecs<T>& V, T alpha,
                                                T beta, double* out, const Grid& g) {
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::N;
  const int64_t n = S.n;
  const int64_t nv = n / VN;
  VT* x = reinterpret_cast<VT*>(V.xh);
  VT* p = reinterpret_cast<VT*>(V.p);
  const VT* r = reinterpret_cast<const VT*>(V.r);
  const VT* sc = reinterpret_cast<const VT*>(S.disq);
  for (int64_t iv = g.gtid; iv < nv; iv += g.gstride) {
    VT xv = x[iv], pv = p[iv], rv, dv;
    if (!FINAL) rv = r[iv];
    if (FINAL && JAC) dv = __ldg(sc + iv);
#pragma unroll
    for (int j = 0; j < VN; ++j) {
      const T pj = lane<T>(pv, j);
      const T xj = fma(alpha, pj, lane<T>(xv, j));
      if (FINAL) {
        const T xo = JAC ? xj * lane<T>(dv, j) : xj;
        if (OUT_ADD) out[iv * VN + j] += (double)xo;
        else out[iv * VN + j] = (double)xo;
      } else {
        lane<T>(xv, j) = xj;
        lane<T>(pv, j) = fma(beta, pj, lane_c<T>(rv, j));
      }
    }
    if (!FINAL) {
      x[iv] = xv;
      p[iv] = pv;
    }
  }
  for (int64_t i = nv * VN + g.gtid; i < n; i += g.gstride) {
    const T pj = V.p[i];
    const T xj = fma(alpha, pj, V.xh[i]);
    if (FINAL) {
      const T xo = JAC ? xj * __ldg(S.disq + i) : xj;
      if (OUT_ADD) out[i] += (double)xo;
      else out[i] = (double)xo;
    } else {
      V.xh[i] = xj;
      V.p[i] = fma(beta, pj, V.r[i]);
    }
  }
}

// The CG loop of Alg. 1 on the loop matrix from a (re)start state: r^ set,
// p = r^, x^ set, rho = r^.r^, rr = the true-norm r.r.  Iterates until
// sqrt(rr) <= stop_abs (kOk), maxit SpMVs (kNotConverged), breakdown /
// non-finite (kBreakdown / kNumeric) or a barrier timeout (kTimeout); *iters
// advances by the SpMVs done.  When an iteration ran, the caller's x is
// written (out = scale x^, or out += fl64(scale x^) with OUT_ADD) before the
// final grid barrier; otherwise out keeps its exact value.
template <typename T, bool JAC, bool OUT_ADD>
__device__ int cg_loop(const Sell<T>& S, const LoopVecs<T>& V, double rho, double rr,
                       double stop_abs, int maxit, int* iters, double* rr_out, double* out,
                       double* part, int pstride, Grid& g, PhaseClock& clk,
                       double* rho_last = nullptr) {
  constexpr bool kExact = sizeof(T) == 4;  // the fp64 loop keeps the fp64 sums (register budget)
  if (rho_last) *rho_last = rho;  // r.z before the last step taken (reliable updates)
  int k = *iters;
  int status = kNotConverged;
  const double stop2_hi = stop2_high(stop_abs);
  bool done = sqrt(rr) <= stop_abs || k >= maxit;  // a4: tested before every SpMV
  if (sqrt(rr) <= stop_abs) status = kOk;
  while (!done) {
    // a1: q = A^ p; p.q
    double v1[1] = {spmv_phase<T, JAC>(S, V.p, V.q, g)};
    publish<1, kExact>(v1, part + kSlotPQ * (size_t)pstride, g);
    clk.lap(g.st, 0);
    if (!g.sync()) { status = kTimeout; break; }
    clk.lap(g.st, 1);
    double pq[1];
    grid_sum<1, kExact>(part + kSlotPQ * (size_t)pstride, g.G, pq);
    // scalars once per CTA in thread 0, shared (fp64 divisions and tests in every
    // thread would load GB300's narrow fp64 pipe)
    __shared__ double s_sc[3];
    __shared__ int s_fl[2];
    if (threadIdx.x == 0) {
      s_fl[0] = (!isfinite(pq[0]) || !isfinite(rho)) ? kNumeric : (pq[0] <= 0.0 ? kBreakdown : 0);
      s_sc[0] = rho / pq[0];
      s_fl[1] = JAC && rr_wanted(S, rho, stop_abs * stop_abs);
    }
    __syncthreads();
    if (s_fl[0]) { status = s_fl[0]; break; }
    const T alpha = (T)s_sc[0];
    // a2: r^ -= alpha q; r.z, r.r (r.r only when the test needs it)
    const bool want_rr = s_fl[1] != 0;
    double v2[2] = {0.0, 0.0};
    update_r_phase<T, JAC>(S, V, alpha, want_rr, v2[0], v2[1], g);
    publish<2, kExact>(v2, part + kSlotUpd * (size_t)pstride, g);
    clk.lap(g.st, 2);
    if (!g.sync()) { status = kTimeout; break; }
    clk.lap(g.st, 3);
    double s2[2];
    grid_sum<2, kExact>(part + kSlotUpd * (size_t)pstride, g.G, s2);
    if (threadIdx.x == 0) {
      double rr_ = s2[1];
      s_sc[1] = s2[0] / rho;
      s_fl[0] = JAC && !want_rr && rr_bound_test(S, s2[0], stop_abs * stop_abs, &rr_) < 0;
      s_sc[2] = rr_;
    }
    __syncthreads();
    const T beta = (T)s_sc[1];
    if (rho_last) *rho_last = rho;
    rho = s2[0];
    rr = s_sc[2];
    if (s_fl[0]) {
      double v3[1] = {rr_phase<T>(S, V, g)};  // rho fell into the band early: exact r.r
      publish<1, kExact>(v3, part + kSlotRr * (size_t)pstride, g);
      if (!g.sync()) { status = kTimeout; break; }
      grid_sum<1, kExact>(part + kSlotRr * (size_t)pstride, g.G, v3);
      rr = v3[0];
    }
    ++k;
    if (threadIdx.x == 0) s_fl[1] = below_stop(rr, stop_abs, stop2_hi);
    __syncthreads();
    const bool conv = s_fl[1] != 0;
    done = conv || k >= maxit;
    if (conv) status = kOk;
    // a3: x^ += alpha p; p = r^ + beta p (last iteration: write the caller's x)
    if (done) update_xp_phase<T, JAC, true, OUT_ADD>(S, V, alpha, beta, out, g);
    else update_xp_phase<T, JAC, false, OUT_ADD>(S, V, alpha, beta, out, g);
    clk.lap(g.st, 4);
    if (!g.sync()) { status = kTimeout; break; }
    clk.lap(g.st, 5);
  }
  *iters = k;
  *rr_out = rr;
  if (status == kNumeric || status == kBreakdown) {
    // the caller's x gets the last iterate
    for (int64_t i = g.gtid; i < S.n; i += g.gstride) {
      const T xo = JAC ? V.xh[i] * __ldg(S.disq + i) : V.xh[i];
      if (OUT_ADD) out[i] += (double)xo;
      else out[i] = (double)xo;
    }
    if (!g.sync()) return kTimeout;
  }
  return status;
}

// Caller's-matrix SpMV q = A x over the original row blocks (a5, restarts,
// the refinement's fp64 residual): the row-block kernel of cg_spmv (one fused
// multiply-add per nonzero in storage order, half the fp64 instructions of a
// separate multiply and add on GB300's narrow fp64 pipe).
__device__ __forceinline__ void spmv_orig(const Csr<double>& A, const double* x, double* q, const Grid& g) {
  __shared__ __align__(16) int s_col[kCap];
  __shared__ __align__(16) double s_val[kCap];
  __shared__ int s_med[kBlock];
  __shared__ int s_nmed;
  for (int b = (int)g.cta; b < A.nrb; b += (int)g.G) spmv_rowblock_fma(A, x, q, b, s_col, s_val, s_med, &s_nmed);
}

// fp64 (Jacobi-)PCG with true-residual check and residual-replacement
// restarts (readings R1-R5 of the method, see the oracle's header).
template <bool JAC>
__global__ void __launch_bounds__(kBlock, 2) pcg64_kernel(SolveParams P) {
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  PhaseClock clk(P.timers != 0);
  const int64_t n = P.A.n;
  const LoopVecs<double>& V = P.V64;
  int status = kNotConverged, k = 0, restarts = 0;
  double relres_true = 0.0, rr = 0.0, bb = 0.0;
  bool first = true;
  for (;;) {
    // a5 / (re)start: r = b - A x; r^ = D^-1/2 r; x^ = D^1/2 x
    spmv_orig(P.A, P.x, V.q, g);
    if (!g.sync()) { status = kTimeout; break; }
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t i = g.gtid; i < n; i += g.gstride) {
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
    publish<3, false>(v, P.part + kSlotRes * (size_t)P.pstride, g);
    if (!g.sync()) { status = kTimeout; break; }
    double s3[3];
    grid_sum<3, false>(P.part + kSlotRes * (size_t)P.pstride, g.G, s3);
    if (first) {
      bb = s3[2];
      if (bb == 0.0) {  // b = 0: x = 0 solves it
        for (int64_t i = g.gtid; i < n; i += g.gstride) P.x[i] = 0.0;
        status = kOk;
        break;
      }
    } else {
      relres_true = sqrt(s3[1]) / sqrt(bb);
      if (!isfinite(relres_true)) { status = kNumeric; break; }
      if (relres_true <= P.tol) { status = kOk; break; }
      if (k >= P.maxit || restarts >= P.max_restarts) { status = kNotConverged; break; }
      ++restarts;
    }
    const bool was_first = first;
    first = false;
    rr = s3[1];
    const int k_before = k;
    const int st = cg_loop<double, JAC, false>(P.S64, V, s3[0], rr, P.tol * sqrt(bb), P.maxit,
                                               &k, &rr, P.x, P.part, P.pstride, g, clk);
    if (st == kTimeout) { status = kTimeout; break; }
    if (st == kNumeric || st == kBreakdown) {
      status = st;
      spmv_orig(P.A, P.x, V.q, g);  // report the true residual of the last iterate
      if (!g.sync()) { status = kTimeout; break; }
      double w[1] = {0.0};
      for (int64_t i = g.gtid; i < n; i += g.gstride) {
        const double ri = P.b[i] - V.q[i];
        w[0] += ri * ri;
      }
      publish<1, false>(w, P.part + kSlotRes * (size_t)P.pstride, g);
      if (!g.sync()) { status = kTimeout; break; }
      double s1[1];
      grid_sum<1, false>(P.part + kSlotRes * (size_t)P.pstride, g.G, s1);
      relres_true = sqrt(s1[0]) / sqrt(bb);
      break;
    }
    if (was_first && k == k_before && st == kOk) {  // x0 met tol: its true residual is s3[1]
      relres_true = sqrt(s3[1]) / sqrt(bb);
      status = kOk;
      break;
    }
    // kOk or kNotConverged: loop back to recompute the true residual
  }
  // CTA 0 reports; a timeout anywhere is visible to the host through st->abort
  if (g.cta == 0 && threadIdx.x == 0) {
    P.st->status = status;
    P.st->iters = k;
    P.st->restarts = restarts;
    P.st->relres_true = relres_true;
    P.st->relres_rec = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
  }
}

// fp32-inner / fp64-outer iterative refinement (reading R6): the outer fp64
// residual, solution update and convergence test, the inner fp32 (scaled
// Jacobi) CG with fp64-accumulated dot products, all in one launch.  CARRY
// (reliable updates, R8): after each fp64 update the inner CG continues from
// the replaced residual with its last search direction, p = r^' + (r^'.r^' /
// rho_k) p_k, instead of restarting from p = r^'.
template <bool JAC, bool CARRY>
__global__ void __launch_bounds__(kBlock, 2) pcg_ir_kernel(SolveParams P) {
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  PhaseClock clk(P.timers != 0);
  const int64_t n = P.A.n;
  const LoopVecs<float>& V = P.V32;
  int status = kNotConverged, inner = 0, outer = 0;
  double relres = 0.0, bb = 0.0, rr32 = 0.0, rho_k = 0.0;
  for (;;) {
    // outer fp64 residual r = b - A x fused with the inner start:
    // r^32 = fl32(D^-1/2 r), d^ = 0
    spmv_orig(P.A, P.x, P.V64.q, g);
    if (!g.sync()) { status = kTimeout; break; }
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = g.gtid; i < n; i += g.gstride) {
      const double bi = P.b[i];
      const double ri = bi - P.V64.q[i];
      const float rh = (float)(JAC ? ri * __ldg(P.disq + i) : ri);
      V.r[i] = rh;
      if (!CARRY || outer == 0) V.p[i] = rh;
      V.xh[i] = 0.0f;
      const double rh2 = (double)rh * (double)rh;
      v[0] += ri * ri;
      v[1] += bi * bi;
      v[2] += rh2;
      v[3] += JAC ? (double)__ldg(P.S32.dn + i) * rh2 : rh2;
    }
    publish<4>(v, P.part + kSlotRes * (size_t)P.pstride, g);
    if (!g.sync()) { status = kTimeout; break; }
    double s4[4];
    grid_sum<4>(P.part + kSlotRes * (size_t)P.pstride, g.G, s4);
    if (outer == 0) {
      bb = s4[1];
      if (bb == 0.0) {
        for (int64_t i = g.gtid; i < n; i += g.gstride) P.x[i] = 0.0;
        status = kOk;
        break;
      }
    }
    relres = sqrt(s4[0]) / sqrt(bb);
    if (!isfinite(relres)) { status = kNumeric; break; }
    if (relres <= P.tol) { status = kOk; break; }
    if (outer >= P.max_restarts || inner >= P.maxit) { status = kNotConverged; break; }
    if (CARRY && outer > 0 && rho_k > 0.0) {  // p = r^' + beta p_k
      const float beta = (float)(s4[2] / rho_k);
      for (int64_t i = g.gtid; i < n; i += g.gstride) V.p[i] = fma(beta, V.p[i], V.r[i]);
      if (!g.sync()) { status = kTimeout; break; }
    }
    const int st = cg_loop<float, JAC, true>(P.S32, V, s4[2], s4[3], P.tol_in * sqrt(s4[3]),
                                             P.maxit, &inner, &rr32, P.x, P.part, P.pstride, g, clk,
                                             &rho_k);
    if (st == kTimeout || st == kNumeric || st == kBreakdown) { status = st; break; }
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

}  // namespace cg
