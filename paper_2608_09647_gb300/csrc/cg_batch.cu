// Batched solves: up to CG_BATCH_MAX_SYSTEMS independent SPD systems of
// uneven size in one persistent cooperative launch, captured in a CUDA graph.
// Each system follows the single-system method of cg_solve (CG / Jacobi-PCG
// of Sec. 3 with its stopping rule, true-residual check and restarts); only
// the schedule is shared.
//
// Layout.  The systems are concatenated into one block-diagonal loop matrix
// of 32-row slices stored column-major (the diagonal held apart as a vector;
// with Jacobi the matrix is the scaled D^-1/2 A D^-1/2 of unit diagonal): a
// system whose off-diagonal entries lie on at most kBatchDiag offsets is
// stored by diagonal (a slot per offset, the gather index clamped into the
// system's own rows, no column array), the others as SELL-32 with global
// columns.  Every system is padded to whole 256-row tiles (padding rows are
// identity rows with b = x = 0), so no tile spans two systems; 16 tiles form a
// 4096-row reduction group.
//
// Schedule.  Rounds of four phases separated by bounded grid barriers:
//   R  r = b - A x for the systems that need it (start, after their loop,
//      restarts): the fp64 true-residual test and the start of a loop;
//   A  q = A p and p.q, alpha;
//   B  r -= alpha q, r.r and r.D r, beta and the recursive stopping test;
//   C  x += alpha p, p = r + beta p.
// A system's stage says which phases it takes part in: 0 residual pending,
// 1 iterating, 2 done, 3 last x update pending (C, then R), 4 r.D r pending.
// At the start of each phase every CTA scans the stages, forms the prefix sum
// of the work of the systems in that phase in shared memory (a unit per
// group, or in the SpMV phases R and A a row-cost weight per group) and takes
// a contiguous chunk of it, so finished systems cost nothing and a chunk
// spans few systems.  A system's sums are formed by the CTA that completes
// its last group of the phase, over (group, warp) partials in order, so they
// do not depend on the schedule.  A stage change made during a phase carries
// that phase's number; a CTA that reads the word in the same phase takes the
// stage from before the change, so all CTAs deal the same list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cg_handle.cuh"

using namespace cg;

namespace {

constexpr int kTile = kBlock;        // rows per tile (kWarps slices, one per warp)
constexpr int kGroup = 16;           // tiles per reduction group (4096 rows)
constexpr int kMaxBatch = CG_BATCH_MAX_SYSTEMS;
constexpr int kNP = 4;               // partial sums per (group, warp)
constexpr int kBatchDiag = 8;        // offsets of a system in the diagonal layout, at most
constexpr int kStRunning = 100;      // status of a system still being solved
constexpr int kMaxCand = 8;          // autotuner candidates
constexpr double kRrMarginB = 64.0;  // r.D r is computed while dmin r^.r^ <= 64 stop^2

// stages and the phases that take them
constexpr int kStResidual = 0, kStIter = 1, kStDone = 2, kStLastX = 3, kStRrPending = 4;
constexpr unsigned kMaskR = (1u << kStResidual) | (1u << kStLastX);
constexpr unsigned kMaskAB = 1u << kStIter;
constexpr unsigned kMaskC = (1u << kStIter) | (1u << kStLastX) | (1u << kStRrPending);
constexpr unsigned kMaskAlive = ~(1u << kStDone);

struct BatchParams {
  int nsys;
  const int32_t* __restrict__ tstart;  // first tile of each system
  const int32_t* __restrict__ ntile;   // tiles of each system
  const int32_t* __restrict__ gstart;  // first reduction group of each system
  const int32_t* __restrict__ ngroup;  // reduction groups of each system
  const int32_t* __restrict__ wcost;   // SpMV-phase cost of a row of each system (load balance)
  const int32_t* __restrict__ sdia;    // offsets of each system in the diagonal layout (0: sliced ELL)
  const int32_t* __restrict__ sdelta;  // those offsets, kBatchDiag per system
  const double* __restrict__ dmin;     // smallest A_ii of each system
  const int32_t* __restrict__ soff;    // slice offsets (units of 32 entries)
  const int32_t* __restrict__ col;     // global (concatenated) column of each entry
  const double* __restrict__ val;
  const double* __restrict__ dg;       // A_ii, 1 on padding rows
  double *r, *p, *q, *xh;
  const double* __restrict__ bh;
  double *rho, *rr, *bb, *alpha, *beta, *relres;
  int *k, *restarts, *status, *zero, *wrr;
  unsigned long long* sstate;          // phase << 16 | stage before << 8 | stage after
  unsigned* cnt;                       // groups of the system finished in this phase
  double* tpart;                       // kNP partials per (group, warp)
  double tol;
  int maxit, max_restarts;
  DevState* st;
  uint64_t timeout_ns;
  unsigned skip_seq;
  // fp32 inner solves with fp64 refinement (batch_ir_kernel only)
  const float* __restrict__ val32;     // the loop matrix values rounded to fp32
  float *r32, *p32, *q32, *d32;        // inner residual, direction, A p, correction d
  double* rho_k;                       // r.z before the last step of the inner solve
  double* beta0;                       // carry factor of the inner solve being started
  double* stopin;                      // inner stopping threshold tol_in ||r32|| (true norm)
  int* start;                          // 1: the A and B phases begin an inner solve
  double tol_in;
  int max_outer, carry;
};

__device__ __forceinline__ int eff_stage(unsigned long long w, unsigned seq) {
  return ((unsigned)(w >> 16) == seq) ? (int)((w >> 8) & 0xff) : (int)(w & 0xff);
}

// Exclusive prefix sum (in s_pref) of the work units of the systems whose
// stage, as seen in phase seq, is in `mask` (a unit per reduction group, or
// WEIGHTED: wcost units per group, the SpMV phases' row cost); returns their
// total.
// *alive gets whether any system is still unfinished.  Thread t owns a
// contiguous run of systems; the runs' totals are scanned with warp shuffles.
template <bool WEIGHTED>
__device__ int build_list(const BatchParams& P, unsigned mask, unsigned seq, int* s_pref, int* s_warp,
                          bool* alive) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int per = (P.nsys + kBlock - 1) / kBlock;
  const int s0 = min(P.nsys, t * per), s1 = min(P.nsys, s0 + per);
  int c = 0, live = 0;
  for (int s = s0; s < s1; ++s) {
    const unsigned sbit = 1u << eff_stage(__ldcg(P.sstate + s), seq);
    const int cs = (sbit & mask) ? P.ngroup[s] * (WEIGHTED ? P.wcost[s] : 1) : 0;
    live |= (sbit & kMaskAlive) != 0;
    s_pref[s] = cs;
    c += cs;
  }
  int inc = c;  // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_warp[warp] = inc;
  *alive = __syncthreads_or(live) != 0;
  int wbase = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const int v = s_warp[w];
    wbase += w < warp ? v : 0;
    total += v;
  }
  int base = wbase + inc - c;
  for (int s = s0; s < s1; ++s) {
    const int cs = s_pref[s];
    s_pref[s] = base;
    base += cs;
  }
  __syncthreads();
  return total;
}

// The system owning entry j of the phase's list: the last system whose
// prefix is <= j (systems without groups in the phase share the prefix of
// their successor, which is larger than j).
__device__ __forceinline__ int system_of(const BatchParams& P, const int* s_pref, int j) {
  int lo = 0, hi = P.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_pref[mid] <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// acc + off-diagonal part of one row of slice sl: the sum over the slice
// width of val * v[col], all loads of a slice issued together (widths 4 and
// 8, those of the 5- and 9-point stencils, unrolled exactly).
template <int W>
__device__ __forceinline__ double slice_row(const int32_t* __restrict__ cp, const double* __restrict__ vp,
                                            const double* __restrict__ v, double acc) {
  int c[W];
  double a[W];
#pragma unroll
  for (int m = 0; m < W; ++m) {
    c[m] = ld_stream(cp + m * 32);
    a[m] = ld_stream(vp + m * 32);
  }
#pragma unroll
  for (int m = 0; m < W; ++m) acc = fma(a[m], v[c[m]], acc);
  return acc;
}

// The system a CTA's current segment belongs to, as row_spmv needs it
// (shared memory, written by run_phase at the start of each segment).
struct SegInfo {
  int nd;              // offsets of the diagonal layout (0: sliced ELL)
  int lo, hi;          // the system's first and last concatenated rows
  int delta[kBatchDiag];
};

// Diagonal layout: column i + delta[m], clamped into the system's own rows
// (the value is 0 there, and no other system's vector is read).
template <int W>
__device__ __forceinline__ double slice_row_dia(const double* __restrict__ vp, const double* __restrict__ v,
                                                int i, const SegInfo& sg, double acc) {
  double a[W], x[W];
#pragma unroll
  for (int m = 0; m < W; ++m) {
    a[m] = ld_stream(vp + m * 32);
    x[m] = v[min(max(i + sg.delta[m], sg.lo), sg.hi)];
  }
#pragma unroll
  for (int m = 0; m < W; ++m) acc = fma(a[m], x[m], acc);
  return acc;
}

__device__ __forceinline__ double row_spmv(const BatchParams& P, const double* __restrict__ v, int i,
                                           double acc, const SegInfo& sg) {
  const int sl = i >> 5, lane = i & 31;
  const int o0 = __ldg(P.soff + sl);
  const int w = __ldg(P.soff + sl + 1) - o0;
  if (sg.nd) {
    const double* vp = P.val + (int64_t)o0 * 32 + lane;
    if (w == 8) return slice_row_dia<8>(vp, v, i, sg, acc);
    if (w == 4) return slice_row_dia<4>(vp, v, i, sg, acc);
    for (int m = 0; m < w; ++m) acc = fma(ld_stream(vp + m * 32), v[min(max(i + sg.delta[m], sg.lo), sg.hi)], acc);
    return acc;
  }
  const int32_t* cp = P.col + (int64_t)o0 * 32 + lane;
  const double* vp = P.val + (int64_t)o0 * 32 + lane;
  if (w == 8) return slice_row<8>(cp, vp, v, acc);
  if (w == 4) return slice_row<4>(cp, vp, v, acc);
  for (int m0 = 0; m0 < w; m0 += 4) {
    if (m0 + 4 <= w) {
      acc = slice_row<4>(cp + m0 * 32, vp + m0 * 32, v, acc);
    } else {
      for (int m = m0; m < w; ++m) acc = fma(ld_stream(vp + m * 32), v[ld_stream(cp + m * 32)], acc);
    }
  }
  return acc;
}

// The same row sum for any value type TV, accumulator TA and gathered vector:
// gx(j) gives the vector's entry j (the fp32 inner solves gather r + beta0 p on
// the first iteration of an inner solve without storing that vector first).
template <int W, typename TV, typename TA, class Gx>
__device__ __forceinline__ TA slice_row_g(const int32_t* __restrict__ cp, const TV* __restrict__ vp, Gx gx,
                                          TA acc) {
  int c[W];
  TV a[W];
#pragma unroll
  for (int m = 0; m < W; ++m) {
    c[m] = ld_stream(cp + m * 32);
    a[m] = ld_stream(vp + m * 32);
  }
  TA x[W];
#pragma unroll
  for (int m = 0; m < W; ++m) x[m] = gx(c[m]);
#pragma unroll
  for (int m = 0; m < W; ++m) acc = fma((TA)a[m], x[m], acc);
  return acc;
}

template <int W, typename TV, typename TA, class Gx>
__device__ __forceinline__ TA slice_row_dia_g(const TV* __restrict__ vp, Gx gx, int i, const SegInfo& sg, TA acc) {
  TV a[W];
  TA x[W];
#pragma unroll
  for (int m = 0; m < W; ++m) {
    a[m] = ld_stream(vp + m * 32);
    x[m] = gx(min(max(i + sg.delta[m], sg.lo), sg.hi));
  }
#pragma unroll
  for (int m = 0; m < W; ++m) acc = fma((TA)a[m], x[m], acc);
  return acc;
}

template <typename TV, typename TA, class Gx>
__device__ __forceinline__ TA row_spmv_g(const BatchParams& P, const TV* __restrict__ val, int i, TA acc,
                                         const SegInfo& sg, Gx gx) {
  const int sl = i >> 5, lane = i & 31;
  const int o0 = __ldg(P.soff + sl);
  const int w = __ldg(P.soff + sl + 1) - o0;
  const TV* vp = val + (int64_t)o0 * 32 + lane;
  if (sg.nd) {
    if (w == 8) return slice_row_dia_g<8, TV, TA>(vp, gx, i, sg, acc);
    if (w == 4) return slice_row_dia_g<4, TV, TA>(vp, gx, i, sg, acc);
    for (int m = 0; m < w; ++m) acc = fma((TA)ld_stream(vp + m * 32), gx(min(max(i + sg.delta[m], sg.lo), sg.hi)), acc);
    return acc;
  }
  const int32_t* cp = P.col + (int64_t)o0 * 32 + lane;
  if (w == 8) return slice_row_g<8, TV, TA>(cp, vp, gx, acc);
  if (w == 4) return slice_row_g<4, TV, TA>(cp, vp, gx, acc);
  for (int m0 = 0; m0 < w; m0 += 4) {
    if (m0 + 4 <= w) {
      acc = slice_row_g<4, TV, TA>(cp + m0 * 32, vp + m0 * 32, gx, acc);
    } else {
      for (int m = m0; m < w; ++m) acc = fma((TA)ld_stream(vp + m * 32), gx(ld_stream(cp + m * 32)), acc);
    }
  }
  return acc;
}

// Sum of a system's (group, warp) partials in a fixed order, given to every
// thread: thread t adds partials t, t + kBlock, ... in order (its loads four at
// a time, so the whole CTA waits for about one L2 round trip), then cta_sum0.
// It runs in the CTA that completes the system while the others wait at the
// next grid barrier, so its latency is the phase's tail.
constexpr int kSumBatch = 4;
template <int NV>
__device__ __forceinline__ void system_sum(const BatchParams& P, int sys, double (&out)[NV]) {
  __shared__ double s_out[NV];
  const int p0 = P.gstart[sys] * kWarps, np = P.ngroup[sys] * kWarps;
  double a[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) a[j] = 0.0;
  for (int t0 = threadIdx.x; t0 < np; t0 += kBlock * kSumBatch) {
    double v[kSumBatch][NV];
#pragma unroll
    for (int u = 0; u < kSumBatch; ++u) {
      const int t = t0 + kBlock * u;
#pragma unroll
      for (int j = 0; j < NV; ++j) v[u][j] = t < np ? __ldcg(P.tpart + (size_t)(p0 + t) * kNP + j) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kSumBatch; ++u) {
      if (t0 + kBlock * u < np) {
#pragma unroll
        for (int j = 0; j < NV; ++j) a[j] += v[u][j];
      }
    }
  }
  cta_sum0<NV>(a);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) s_out[j] = a[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = s_out[j];
  __syncthreads();
}

// New stage of sys, tagged with the current phase (one writer per system and phase).
__device__ __forceinline__ void set_stage(const BatchParams& P, int sys, int stage, unsigned seq) {
  const unsigned long long before = __ldcg(P.sstate + sys) & 0xffull;
  P.sstate[sys] = ((unsigned long long)seq << 16) | (before << 8) | (unsigned long long)stage;
}

// One phase over its list of reduction groups [0, T).  CTA c takes the
// contiguous chunk [c T / G, (c+1) T / G), which spans few systems.  At the
// start of each system's segment begin(sys) loads the system's scalars and
// says whether its sums are wanted.  For every row i of a group, row(i) does
// the row's loads and arithmetic and returns its commit, which stores the
// results and adds the row's NV contributions to the thread's accumulators.
// A thread's rows go in groups of ROWS (8, 4, 2 or 1, by the variant's register
// budget), every row's loads in flight before the first commit (a store ahead
// of the next row's loads would serialise them); the accumulation order stays
// the row order.  The group's sums are then reduced
// per warp (xor tree) and stored.  Leaving a segment, the CTA adds its group count to the system's
// counter; the CTA that completes the count sums the system's partials in
// (group, warp) order, independent of G, and calls done(sys, sums) in thread 0.
// Sums NREQ.. NV-1 are reduced only while *opt holds (set by begin for the segment's system).
template <int NV, int ROWS, bool WEIGHTED, int NREQ = NV, class Begin, class Row, class Done>
__device__ __forceinline__ void run_phase(const BatchParams& P, const int* s_pref, int T, const Grid& g,
                                          SegInfo& seg, Begin begin, Row row, Done done,
                                          const bool* opt = nullptr) {
  __shared__ int s_last;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int j1 = (int)((int64_t)T * (g.cta + 1) / g.G);
  int j = (int)((int64_t)T * g.cta / g.G);
  while (j < j1) {
    const int sys = system_of(P, s_pref, j);
    // this CTA's groups of sys: those whose first unit lies in [j, j1)
    const int w = WEIGHTED ? P.wcost[sys] : 1;
    const int base = s_pref[sys];
    const int g0 = (j - base + w - 1) / w;
    const int g1 = min(P.ngroup[sys], (j1 - base + w - 1) / w);
    const int next = base + P.ngroup[sys] * w;  // the next system's first unit
    if (g0 >= g1) {
      j = min(j1, next);
      continue;
    }
    if (t == 0) {
      seg.nd = P.sdia[sys];
      seg.lo = P.tstart[sys] * kTile;
      seg.hi = seg.lo + P.ntile[sys] * kTile - 1;
#pragma unroll
      for (int m = 0; m < kBatchDiag; ++m) seg.delta[m] = P.sdelta[sys * kBatchDiag + m];
    }
    __syncthreads();
    const bool sums = begin(sys);
    const int tend = P.tstart[sys] + P.ntile[sys];
    for (int grp = g0; grp < g1; ++grp) {
      const int t0 = P.tstart[sys] + grp * kGroup, t1 = min(t0 + kGroup, tend);
      double acc[NV > 0 ? NV : 1];
#pragma unroll
      for (int k = 0; k < (NV > 0 ? NV : 1); ++k) acc[k] = 0.0;
      int gt = t0;
      if constexpr (ROWS >= 8) {
        for (; gt + 7 < t1; gt += 8) {
          const auto c0 = row(gt * kTile + t);
          const auto c1 = row((gt + 1) * kTile + t);
          const auto c2 = row((gt + 2) * kTile + t);
          const auto c3 = row((gt + 3) * kTile + t);
          const auto c4 = row((gt + 4) * kTile + t);
          const auto c5 = row((gt + 5) * kTile + t);
          const auto c6 = row((gt + 6) * kTile + t);
          const auto c7 = row((gt + 7) * kTile + t);
          c0(acc);
          c1(acc);
          c2(acc);
          c3(acc);
          c4(acc);
          c5(acc);
          c6(acc);
          c7(acc);
        }
      }
      if constexpr (ROWS >= 4) {
        for (; gt + 3 < t1; gt += 4) {
          const auto c0 = row(gt * kTile + t);
          const auto c1 = row((gt + 1) * kTile + t);
          const auto c2 = row((gt + 2) * kTile + t);
          const auto c3 = row((gt + 3) * kTile + t);
          c0(acc);
          c1(acc);
          c2(acc);
          c3(acc);
        }
      }
      if constexpr (ROWS >= 2) {
        for (; gt + 1 < t1; gt += 2) {
          const auto c0 = row(gt * kTile + t);
          const auto c1 = row((gt + 1) * kTile + t);
          c0(acc);
          c1(acc);
        }
      }
      for (; gt < t1; ++gt) row(gt * kTile + t)(acc);
      if (NV > 0 && sums) {
        // the warp's sum of each reduced value, exact and rounded once on the integer
        // pipes: an fp64 xor tree would take 5 warp instructions of the fp64 pipe
        // (one per ~64 clocks per SM sub-partition) that the rows' FMAs need
        const bool all = NREQ >= NV || (opt && *opt);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          if (k < NREQ || all) acc[k] = warp_sum_exact(acc[k]);
        }
        if (lane == 0) {
          double* dst = P.tpart + ((size_t)(P.gstart[sys] + grp) * kWarps + warp) * kNP;
#pragma unroll
          for (int k = 0; k < NV; ++k)
            if (k < NREQ || all) dst[k] = acc[k];
        }
      }
    }
    if (NV > 0 && sums) {
      if (lane == 0) __threadfence();  // partials visible before the count
      __syncthreads();
      if (t == 0) {
        const unsigned add = (unsigned)(g1 - g0);
        const unsigned prev = atomicAdd(P.cnt + sys, add);
        const int last = prev + add == (unsigned)P.ngroup[sys];
        if (last) P.cnt[sys] = 0u;  // reset for the next phase (after its barrier)
        __threadfence();
        s_last = last;
      }
      __syncthreads();
      if (s_last) {
        double sm[NV > 0 ? NV : 1];
        system_sum<NV>(P, sys, sm);
        if (t == 0) done(sys, sm);
      }
    }
    __syncthreads();  // every thread is done with seg before the next segment's
    j = min(j1, next);
  }
}

// MINB: resident CTAs per SM the registers are budgeted for (an autotuner choice).
template <bool JAC, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) batch_pcg_kernel(BatchParams P) {
  // rows in flight per thread within the register budget of MINB CTAs per SM
  constexpr int kRows = MINB <= 3 ? 4 : (MINB == 4 ? 2 : 1);
  // phase B streams only q and r (two loads a row): twice the rows in flight
  constexpr int kRowsB = 2 * kRows;
  __shared__ int s_pref[kMaxBatch];
  __shared__ int s_scan[kWarps];
  __shared__ SegInfo s_seg;
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  double* __restrict__ r = P.r;
  double* __restrict__ p = P.p;
  double* __restrict__ q = P.q;
  double* __restrict__ xh = P.xh;
  const double* __restrict__ bh = P.bh;
  const double* __restrict__ dg = P.dg;
  double c_alpha = 0.0, c_beta = 0.0;  // scalars of the current segment's system
  bool c_flag = false, c_sum = false;
  unsigned seq = 0;  // phase number; the initial stage words carry 0
  for (;;) {
    // ---- R: residual of the stage 0 / 3 systems, their test, (re)start
    ++seq;
    bool alive = false;
    int T = build_list<true>(P, kMaskR, seq, s_pref, s_scan, &alive);
    if (!alive) break;
    if (T > 0) {
      run_phase<3, kRows, true>(
          P, s_pref, T, g, s_seg, [&](int) { return true; },
          [&](int i) {
            const double xi = xh[i];
            const double ri_ax = row_spmv(P, xh, i, JAC ? xi : __ldg(dg + i) * xi, s_seg);
            const double bi = bh[i];
            const double ri = bi - ri_ax;
            const double d = JAC ? __ldg(dg + i) : 1.0;
            return [=](double* acc) {
              r[i] = ri;
              p[i] = ri;
              acc[0] = fma(ri, ri, acc[0]);      // r^.r^ = r.z
              acc[1] = fma(d * ri, ri, acc[1]);  // r.r
              acc[2] = fma(d * bi, bi, acc[2]);  // b.b
            };
          },
          [&](int sys, const double* sm) {
            const bool first = P.bb[sys] < 0.0;
            if (first) P.bb[sys] = sm[2];
            const double bb = P.bb[sys];
            const double rel = bb > 0.0 ? sqrt(sm[1]) / sqrt(bb) : 0.0;
            P.relres[sys] = rel;
            P.rho[sys] = sm[0];
            P.rr[sys] = sm[1];
            P.wrr[sys] = JAC && P.dmin[sys] * sm[0] <= kRrMarginB * P.tol * P.tol * bb;
            int st = P.status[sys], next = kStDone;
            if (bb == 0.0) {
              st = kOk;
              P.zero[sys] = 1;
            } else if (st == kBreakdown || st == kNumeric) {
              // keep: the residual was only wanted for the report
            } else if (!isfinite(rel)) {
              st = kNumeric;
            } else if (rel <= P.tol) {
              st = kOk;
            } else if (P.k[sys] >= P.maxit) {
              st = kNotConverged;
            } else if (first) {
              st = kStRunning;
              next = kStIter;
            } else if (P.restarts[sys] >= P.max_restarts) {
              st = kNotConverged;
            } else {
              P.restarts[sys] += 1;
              st = kStRunning;
              next = kStIter;
            }
            P.status[sys] = st;
            set_stage(P, sys, next, seq);
          });
      if (!g.sync()) return;
    }
    // ---- A: q = A p, alpha
    ++seq;
    T = build_list<true>(P, kMaskAB, seq, s_pref, s_scan, &alive);
    if (T == 0) continue;
    run_phase<1, kRows, true>(
        P, s_pref, T, g, s_seg, [&](int) { return true; },
        [&](int i) {
          const double pi = p[i];
          const double qi = row_spmv(P, p, i, JAC ? pi : __ldg(dg + i) * pi, s_seg);
          return [=](double* acc) {
            q[i] = qi;
            acc[0] = fma(pi, qi, acc[0]);
          };
        },
        [&](int sys, const double* sm) {
          const double rho = P.rho[sys];
          if (!isfinite(sm[0]) || !isfinite(rho)) {
            P.status[sys] = kNumeric;
            set_stage(P, sys, kStResidual, seq);  // residual of the current x, then stop
          } else if (sm[0] <= 0.0) {
            P.status[sys] = kBreakdown;
            set_stage(P, sys, kStResidual, seq);
          } else {
            P.alpha[sys] = rho / sm[0];
          }
        });
    if (!g.sync()) return;
    // ---- B: r -= alpha q, rho' = r^.r^, r.r when near the stopping band, beta, test
    ++seq;
    T = build_list<false>(P, kMaskAB, seq, s_pref, s_scan, &alive);
    run_phase<2, kRowsB, false, 1>(
        P, s_pref, T, g, s_seg,
        [&](int sys) {
          c_alpha = P.alpha[sys];
          c_flag = JAC && P.wrr[sys];
          return true;
        },
        [&](int i) {
          const double ri = fma(-c_alpha, q[i], r[i]);
          const double di = c_flag ? __ldg(dg + i) : 0.0;
          const bool flag = c_flag;
          return [=](double* acc) {
            r[i] = ri;
            acc[0] = fma(ri, ri, acc[0]);
            if (flag) acc[1] = fma(di * ri, ri, acc[1]);
          };
        },
        [&](int sys, const double* sm) {
          const double rho = sm[0];
          P.beta[sys] = rho / P.rho[sys];
          P.rho[sys] = rho;
          const int k = P.k[sys] + 1;
          P.k[sys] = k;
          const double stop2 = P.tol * P.tol * P.bb[sys];
          bool conv;
          if (!JAC || P.wrr[sys]) {
            const double rr = JAC ? sm[1] : rho;
            P.rr[sys] = rr;
            conv = sqrt(rr) <= P.tol * sqrt(P.bb[sys]);
          } else {
            // r.D r >= dmin r^.r^: above the band the test fails for sure
            conv = false;
            if (P.dmin[sys] * rho <= stop2) {
              P.wrr[sys] = 1;
              set_stage(P, sys, kStRrPending, seq);  // exact r.D r in phase C
              return;
            }
          }
          if (JAC) P.wrr[sys] = P.dmin[sys] * rho <= kRrMarginB * stop2;
          if (conv || k >= P.maxit) set_stage(P, sys, kStLastX, seq);
        },
        &c_flag);
    if (!g.sync()) return;
    // ---- C: x += alpha p; p = r + beta p unless the loop ended; pending r.D r
    ++seq;
    T = build_list<false>(P, kMaskC, seq, s_pref, s_scan, &alive);
    run_phase<1, kRows, false>(
        P, s_pref, T, g, s_seg,
        [&](int sys) {
          const int stg = eff_stage(__ldcg(P.sstate + sys), seq);
          c_alpha = P.alpha[sys];
          c_beta = P.beta[sys];
          c_flag = stg != kStLastX;  // p is still needed
          c_sum = stg == kStRrPending;
          return c_sum;
        },
        [&](int i) {
          const double pi = p[i];
          const double xn = fma(c_alpha, pi, xh[i]);
          const double ri = r[i];
          const double pn = fma(c_beta, pi, ri);
          const bool keep_p = c_flag, sum = JAC && c_sum;
          const double di = sum ? __ldg(dg + i) : 0.0;
          return [=](double* acc) {
            xh[i] = xn;
            if (keep_p) p[i] = pn;
            if (sum) acc[0] = fma(di * ri, ri, acc[0]);
          };
        },
        [&](int sys, const double* sm) {
          P.rr[sys] = sm[0];
          const bool conv = sqrt(sm[0]) <= P.tol * sqrt(P.bb[sys]);
          // converged or out of iterations: x is final, so the true residual next
          set_stage(P, sys, conv || P.k[sys] >= P.maxit ? kStResidual : kStIter, seq);
        });
    if (!g.sync()) return;
  }
}

// fp32 inner solves with fp64 refinement (readings R6 and R8 per system).
// Stages beyond the fp64 kernel's: 5 = the step's x/p update is still due (C,
// then iterating), 6 = the inner solve's last update is still due (C, then R).
constexpr int kStCOnly = 5, kStFinalDue = 6;
constexpr unsigned kMaskC32 = (1u << kStIter) | (1u << kStLastX) | (1u << kStRrPending) | (1u << kStCOnly) |
                              (1u << kStFinalDue);

// Every system solved as the single-system refinement solves it: R forms the
// fp64 residual r = b^ - A^ x^ with the fp64 loop matrix, takes the true-residual
// test and starts an inner solve on r32 = fl32(r) (d = 0; with reliable updates,
// P.carry, the search direction carries over: p = r32 + (r32.r32 / rho_k) p_k);
// A, B, C are the inner fp32 PCG on the fp32 loop matrix, sums in fp64, until
// the inner residual has dropped by tol_in; the inner solve's last C phase adds
// fl64(d + alpha p) to x^ and hands the system back to R.  The carried direction
// is never stored before its first use: A gathers r + beta0 p at neighbouring
// rows, and B writes p = r + beta0 p for its own rows before it updates r.
template <bool JAC, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) batch_ir_kernel(BatchParams P) {
  constexpr int kRows = MINB <= 3 ? 4 : (MINB == 4 ? 2 : 1);
  __shared__ int s_pref[kMaxBatch];
  __shared__ int s_scan[kWarps];
  __shared__ SegInfo s_seg;
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  float* __restrict__ r = P.r32;
  float* __restrict__ p = P.p32;
  float* __restrict__ q = P.q32;
  float* __restrict__ d = P.d32;
  double* __restrict__ xh = P.xh;
  const double* __restrict__ bh = P.bh;
  const double* __restrict__ dg = P.dg;
  float c_alpha = 0.0f, c_beta = 0.0f, c_beta0 = 0.0f;
  bool c_flag = false, c_start = false;
  int c_mode = 0;  // C phase: 0 update, 1 last update of the inner solve, 2 r.D r only
  unsigned seq = 0;
  for (;;) {
    // ---- R: fp64 residual, true-residual test, start of an inner solve
    ++seq;
    bool alive = false;
    int T = build_list<true>(P, kMaskR, seq, s_pref, s_scan, &alive);
    if (!alive) break;
    if (T > 0) {
      run_phase<4, kRows, true>(
          P, s_pref, T, g, s_seg, [&](int) { return true; },
          [&](int i) {
            const double xi = xh[i];
            const double ax = row_spmv(P, xh, i, JAC ? xi : __ldg(dg + i) * xi, s_seg);
            const double bi = bh[i];
            const double ri = bi - ax;
            const float r32 = (float)ri;
            const double dd = JAC ? __ldg(dg + i) : 1.0;
            return [=](double* acc) {
              r[i] = r32;
              d[i] = 0.0f;
              const double rs = (double)r32;
              acc[0] = fma(rs, rs, acc[0]);       // r32.r32: the inner rho
              acc[1] = fma(dd * rs, rs, acc[1]);  // r32.D r32: the inner solve's reference norm
              acc[2] = fma(dd * ri, ri, acc[2]);  // fp64 r.r
              acc[3] = fma(dd * bi, bi, acc[3]);  // b.b
            };
          },
          [&](int sys, const double* sm) {
            const bool first = P.bb[sys] < 0.0;
            if (first) P.bb[sys] = sm[3];
            const double bb = P.bb[sys];
            const double rel = bb > 0.0 ? sqrt(sm[2]) / sqrt(bb) : 0.0;
            P.relres[sys] = rel;
            int st = P.status[sys], next = kStDone;
            if (bb == 0.0) {
              st = kOk;
              P.zero[sys] = 1;
            } else if (st == kBreakdown || st == kNumeric) {
              // keep: the residual was only wanted for the report
            } else if (!isfinite(rel)) {
              st = kNumeric;
            } else if (rel <= P.tol) {
              st = kOk;
            } else if (P.k[sys] >= P.maxit || P.restarts[sys] >= P.max_outer || !(sm[0] > 0.0)) {
              st = kNotConverged;  // out of iterations or updates (or r32 underflowed to 0)
            } else {
              const double rho = sm[0];
              P.beta0[sys] = (P.carry && P.rho_k[sys] > 0.0) ? rho / P.rho_k[sys] : 0.0;
              P.rho[sys] = rho;
              P.rr[sys] = sm[1];
              const double stop = P.tol_in * sqrt(sm[1]);
              P.stopin[sys] = stop;
              P.wrr[sys] = JAC && P.dmin[sys] * rho <= kRrMarginB * stop * stop;
              P.start[sys] = 1;
              P.restarts[sys] += 1;  // inner solves started (refinement steps / updates)
              st = kStRunning;
              next = kStIter;
            }
            P.status[sys] = st;
            set_stage(P, sys, next, seq);
          });
      if (!g.sync()) return;
    }
    // ---- A: q = A p (the first step of an inner solve: p = r + beta0 p gathered), alpha
    ++seq;
    T = build_list<true>(P, kMaskAB, seq, s_pref, s_scan, &alive);
    if (T == 0) continue;
    run_phase<1, kRows, true>(
        P, s_pref, T, g, s_seg,
        [&](int sys) {
          c_start = P.start[sys] != 0;
          c_beta0 = (float)P.beta0[sys];
          return true;
        },
        [&](int i) {
          float pi, qi;
          const float dgi = JAC ? 1.0f : (float)__ldg(dg + i);
          if (c_start && c_beta0 != 0.0f) {
            const float b0 = c_beta0;
            auto gx = [=](int j) { return fmaf(b0, p[j], r[j]); };
            pi = gx(i);
            qi = row_spmv_g<float, float>(P, P.val32, i, dgi * pi, s_seg, gx);
          } else if (c_start) {
            auto gx = [=](int j) { return r[j]; };
            pi = r[i];
            qi = row_spmv_g<float, float>(P, P.val32, i, dgi * pi, s_seg, gx);
          } else {
            auto gx = [=](int j) { return p[j]; };
            pi = p[i];
            qi = row_spmv_g<float, float>(P, P.val32, i, dgi * pi, s_seg, gx);
          }
          return [=](double* acc) {
            q[i] = qi;
            acc[0] = fma((double)pi, (double)qi, acc[0]);
          };
        },
        [&](int sys, const double* sm) {
          const double rho = P.rho[sys];
          if (!isfinite(sm[0]) || !isfinite(rho) || sm[0] <= 0.0) {
            // x^ gets the inner iterate so far (d), then R reports its true residual
            P.status[sys] = (!isfinite(sm[0]) || !isfinite(rho)) ? kNumeric : kBreakdown;
            P.alpha[sys] = 0.0;
            set_stage(P, sys, kStLastX, seq);
          } else {
            P.alpha[sys] = rho / sm[0];
          }
        });
    if (!g.sync()) return;
    // ---- B: p = r + beta0 p at the start of an inner solve; r -= alpha q, rho', r.D r near
    //      the band, beta, the inner test
    ++seq;
    T = build_list<false>(P, kMaskAB, seq, s_pref, s_scan, &alive);
    run_phase<2, kRows, false, 1>(
        P, s_pref, T, g, s_seg,
        [&](int sys) {
          c_alpha = (float)P.alpha[sys];
          c_flag = JAC && P.wrr[sys];
          c_start = P.start[sys] != 0;
          c_beta0 = (float)P.beta0[sys];
          return true;
        },
        [&](int i) {
          const float r0 = r[i];
          const float ri = fmaf(-c_alpha, q[i], r0);
          const bool st = c_start;
          const float pn = st ? (c_beta0 != 0.0f ? fmaf(c_beta0, p[i], r0) : r0) : 0.0f;
          const double di = c_flag ? __ldg(dg + i) : 0.0;
          const bool flag = c_flag;
          return [=](double* acc) {
            r[i] = ri;
            if (st) p[i] = pn;
            const double rd = (double)ri;
            acc[0] = fma(rd, rd, acc[0]);
            if (flag) acc[1] = fma(di * rd, rd, acc[1]);
          };
        },
        [&](int sys, const double* sm) {
          P.start[sys] = 0;
          const double rho = sm[0];
          P.beta[sys] = rho / P.rho[sys];
          P.rho_k[sys] = P.rho[sys];  // r.z of the step just taken (the carry's denominator)
          P.rho[sys] = rho;
          const int k = P.k[sys] + 1;
          P.k[sys] = k;
          const double stop = P.stopin[sys];
          bool conv;
          if (!JAC || P.wrr[sys]) {
            const double rr = JAC ? sm[1] : rho;
            P.rr[sys] = rr;
            conv = sqrt(rr) <= stop;
          } else {
            conv = false;  // r.D r >= dmin r^.r^: above the band the test fails for sure
            if (P.dmin[sys] * rho <= stop * stop) {
              P.wrr[sys] = 1;
              set_stage(P, sys, kStRrPending, seq);  // exact r.D r in phase C, no update yet
              return;
            }
          }
          if (JAC) P.wrr[sys] = P.dmin[sys] * rho <= kRrMarginB * stop * stop;
          if (conv || k >= P.maxit) set_stage(P, sys, kStLastX, seq);
        },
        &c_flag);
    if (!g.sync()) return;
    // ---- C: d += alpha p, p = r + beta p; the inner solve's last update x^ += fl64(d + alpha p)
    //      (p stays the last direction); a pending exact r.D r
    ++seq;
    T = build_list<false>(P, kMaskC32, seq, s_pref, s_scan, &alive);
    run_phase<1, kRows, false>(
        P, s_pref, T, g, s_seg,
        [&](int sys) {
          const int stg = eff_stage(__ldcg(P.sstate + sys), seq);
          c_alpha = (float)P.alpha[sys];
          c_beta = (float)P.beta[sys];
          c_mode = (stg == kStLastX || stg == kStFinalDue) ? 1 : (stg == kStRrPending ? 2 : 0);
          // sums (and so done()) for the r.D r pass and to move the deferred stages on
          return stg == kStRrPending || stg == kStCOnly || stg == kStFinalDue;
        },
        [&](int i) {
          const int mode = c_mode;
          // alpha = 0 (a breakdown at an inner solve's first step): p is not read
          const float pi = (mode != 2 && c_alpha != 0.0f) ? p[i] : 0.0f;
          const float di = mode != 2 ? d[i] : 0.0f;
          const float ri = mode != 1 ? r[i] : 0.0f;
          const double xo = mode == 1 ? xh[i] : 0.0;
          const float dn = fmaf(c_alpha, pi, di);
          const float pn = fmaf(c_beta, pi, ri);
          const double dgi = (JAC && mode == 2) ? __ldg(dg + i) : 0.0;
          return [=](double* acc) {
            if (mode == 0) {
              d[i] = dn;
              p[i] = pn;
            } else if (mode == 1) {
              xh[i] = xo + (double)dn;
            } else {
              const double rd = (double)ri;
              acc[0] = fma(JAC ? dgi * rd : rd, rd, acc[0]);
            }
          };
        },
        [&](int sys, const double* sm) {
          const int stg = eff_stage(__ldcg(P.sstate + sys), seq);
          if (stg == kStRrPending) {
            P.rr[sys] = sm[0];
            const bool conv = sqrt(sm[0]) <= P.stopin[sys];
            set_stage(P, sys, conv || P.k[sys] >= P.maxit ? kStFinalDue : kStCOnly, seq);
          } else if (stg == kStCOnly) {
            set_stage(P, sys, kStIter, seq);
          } else {  // kStFinalDue: the last update is done, the fp64 residual is next
            set_stage(P, sys, kStLastX, seq);
          }
        });
    if (!g.sync()) return;
  }
}

// Inner-solve state of every system at the start of an fp32 solve (no direction to carry yet).
__global__ void batch_init_f32_kernel(int nsys, double* rho_k, int* start) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    rho_k[s] = 0.0;
    start[s] = 0;
  }
}

// Per-system copies into the concatenated vectors: b^ = D^-1/2 b, x^ = D^1/2 x
// with Jacobi (b, x unchanged without); zeros on padding rows.
__global__ void batch_gather_kernel(const double* const* b, const double* const* x, const int64_t* n,
                                    const int64_t* r0, const int32_t* ntile, const double* disq,
                                    const double* dsq, int jac, double* bh, double* xh) {
  const int s = blockIdx.y;
  const int64_t ns = n[s], base = r0[s], npad = (int64_t)ntile[s] * kTile;
  const double* bs = b[s];
  const double* xs = x[s];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gi = base + i;
    if (i < ns) {
      bh[gi] = jac ? bs[i] * disq[gi] : bs[i];
      xh[gi] = jac ? xs[i] * dsq[gi] : xs[i];
    } else {
      bh[gi] = 0.0;
      xh[gi] = 0.0;
    }
  }
}

// x = D^-1/2 x^ (x^ without Jacobi) back into the caller's vectors; x = 0 for b = 0.
__global__ void batch_scatter_kernel(double* const* x, const int64_t* n, const int64_t* r0,
                                     const double* disq, int jac, const double* xh, const int* zero) {
  const int s = blockIdx.y;
  const int64_t ns = n[s], base = r0[s];
  double* xs = x[s];
  const bool z = zero[s] != 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gi = base + i;
    xs[i] = z ? 0.0 : (jac ? xh[gi] * disq[gi] : xh[gi]);
  }
}

// Loop state of every system at the start of a solve.
__global__ void batch_init_kernel(int nsys, double* bb, int* k, int* restarts, int* status, int* zero,
                                  int* wrr, unsigned long long* sstate, unsigned* cnt) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    bb[s] = -1.0;  // "not yet known": the first residual phase records b.b
    k[s] = 0;
    restarts[s] = 0;
    status[s] = kStRunning;
    zero[s] = 0;
    wrr[s] = 0;
    sstate[s] = 0ull;  // stage 0, phase 0
    cnt[s] = 0u;
  }
}

// One system's rows into the concatenated slices (thread per padded row):
// off-diagonal entries of row i in storage order, then padding (column = the
// row itself, value 0) up to the slice width.  With SCALE the values are
// A_ij / sqrt(A_ii A_jj), the two scales multiplied first so the scaled
// matrix stays bitwise symmetric when A is.  col may be null (written with
// the other value variant).
template <bool SCALE>
__global__ void batch_fill_kernel(int64_t n, int64_t npad, int64_t r0, int64_t sl0,
                                  const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                  const double* __restrict__ vals, const double* __restrict__ ldisq,
                                  const int32_t* __restrict__ soff, int32_t* col, double* val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = sl0 + (i >> 5), l = i & 31;
    const int64_t base = (int64_t)soff[sl] * 32 + l;
    const int w = soff[sl + 1] - soff[sl];
    int m = 0;
    if (i < n) {
      const double si = SCALE ? ldisq[i] : 1.0;
      for (int k = rowptr[i]; k < rowptr[i + 1] && m < w; ++k) {
        const int c = colind[k];
        if ((int64_t)c == i) continue;
        if (col) col[base + (int64_t)m * 32] = (int32_t)(r0 + c);
        val[base + (int64_t)m * 32] = SCALE ? vals[k] * (si * ldisq[c]) : vals[k];
        ++m;
      }
    }
    for (; m < w; ++m) {
      if (col) col[base + (int64_t)m * 32] = (int32_t)(r0 + i);
      val[base + (int64_t)m * 32] = 0.0;
    }
  }
}

// The diagonal layout of one system (thread per padded row): slot m of row i
// holds the sum of the row's entries in column i + delta[m] (0 where there is
// none, and on padding rows), scaled as batch_fill_kernel does.
struct BatchDelta {
  int nd;
  int d[kBatchDiag];
};
template <bool SCALE>
__global__ void batch_fill_dia_kernel(int64_t n, int64_t npad, int64_t sl0, const int32_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ colind, const double* __restrict__ vals,
                                      const double* __restrict__ ldisq, const int32_t* __restrict__ soff,
                                      BatchDelta bd, double* val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = (int64_t)soff[sl0 + (i >> 5)] * 32 + (i & 31);
    double v[kBatchDiag];
#pragma unroll
    for (int m = 0; m < kBatchDiag; ++m) v[m] = 0.0;
    if (i < n) {
      const double si = SCALE ? ldisq[i] : 1.0;
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int c = colind[k];
        if ((int64_t)c == i) continue;
        const int o = (int)(c - i);
#pragma unroll
        for (int m = 0; m < kBatchDiag; ++m)
          if (m < bd.nd && bd.d[m] == o) v[m] += SCALE ? vals[k] * (si * ldisq[c]) : vals[k];
      }
    }
#pragma unroll
    for (int m = 0; m < kBatchDiag; ++m)
      if (m < bd.nd) val[base + (int64_t)m * 32] = v[m];
  }
}

// Diagonal vectors of one system at its rows of the concatenation: A_ii,
// sqrt(A_ii), 1/sqrt(A_ii) (1 on padding rows and where A_ii <= 0, which
// only the unpreconditioned solve accepts).
__global__ void batch_diag_kernel(int64_t n, int64_t npad, int64_t r0, const double* __restrict__ diag,
                                  double* gd, double* gdsq, double* gdisq) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = i < n ? diag[i] : 1.0;
    const bool pos = d > 0.0;
    const double s = pos ? sqrt(d) : 1.0;
    gd[r0 + i] = d;
    gdsq[r0 + i] = s;
    gdisq[r0 + i] = pos ? 1.0 / s : 1.0;
  }
}

// Kernel variants the autotuner chooses from: registers budgeted for 3, 4 or 5
// resident CTAs per SM (more CTAs hide more memory latency; fewer registers
// may spill).
constexpr int kVariants = 3;
constexpr int kVariantMinBlocks[kVariants] = {3, 4, 5};

const void* batch_kernel(bool jac, int variant, bool f32) {
  if (f32) {
    switch (variant) {
      case 0: return jac ? (const void*)batch_ir_kernel<true, 3> : (const void*)batch_ir_kernel<false, 3>;
      case 1: return jac ? (const void*)batch_ir_kernel<true, 4> : (const void*)batch_ir_kernel<false, 4>;
      default: return jac ? (const void*)batch_ir_kernel<true, 5> : (const void*)batch_ir_kernel<false, 5>;
    }
  }
  switch (variant) {
    case 0: return jac ? (const void*)batch_pcg_kernel<true, 3> : (const void*)batch_pcg_kernel<false, 3>;
    case 1: return jac ? (const void*)batch_pcg_kernel<true, 4> : (const void*)batch_pcg_kernel<false, 4>;
    default: return jac ? (const void*)batch_pcg_kernel<true, 5> : (const void*)batch_pcg_kernel<false, 5>;
  }
}

// fp32 copy of the loop matrix values (the same rounding as the single-system
// loop: the scaled fp64 value rounded once).
__global__ void batch_to_f32_kernel(int64_t count, const double* __restrict__ v, float* __restrict__ w) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
    w[k] = (float)v[k];
}

// The autotuner's records and the kernels: one slot per (preconditioner, precision kind).
inline int tune_slot(bool jac, bool f32) { return (jac ? 1 : 0) + (f32 ? 2 : 0); }

unsigned blocks_for(int64_t items) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 4096));
}

}  // namespace

// Device memory of a batch (owned by its cg_handle).
struct BatchData {
  int nsys = 0;
  std::vector<cg_handle*> sys;     // per-system handles (validation, diagonal)
  std::vector<int64_t> n, r0;      // rows and first concatenated row of each system
  std::vector<int32_t> tstart, ntile;
  int64_t rows = 0;                // padded rows in all
  int ntiles = 0, nslices = 0;
  int64_t entries = 0;             // slice entries (multiple of 32)
  int32_t *d_tstart = nullptr, *d_ntile = nullptr, *soff = nullptr, *col = nullptr;
  int32_t *d_gstart = nullptr, *d_ngroup = nullptr, *d_wcost = nullptr;
  std::vector<int32_t> sdia, sdelta;  // diagonal layout of each system and its offsets (kBatchDiag each)
  int32_t *d_sdia = nullptr, *d_sdelta = nullptr;
  int ngroups = 0;                 // reduction groups in all
  double* d_dmin = nullptr;        // smallest A_ii per system
  int64_t *d_n = nullptr, *d_r0 = nullptr;
  double* val[2] = {nullptr, nullptr};  // [precond]: unscaled / Jacobi-scaled
  float* val32[2] = {nullptr, nullptr}; // fp32 copies (fp32 precisions)
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;  // inner fp32 vectors
  double *rho_k = nullptr, *beta0 = nullptr, *stopin = nullptr;          // per system (fp32)
  int* start = nullptr;
  double *dg = nullptr, *dsq = nullptr, *disq = nullptr;
  double *r = nullptr, *p = nullptr, *q = nullptr, *xh = nullptr, *bh = nullptr;
  double *rho = nullptr, *rr = nullptr, *bb = nullptr, *alpha = nullptr, *beta = nullptr,
         *relres = nullptr;
  int *k = nullptr, *restarts = nullptr, *status = nullptr, *zero = nullptr, *wrr = nullptr;
  unsigned long long* sstate = nullptr;
  unsigned* cnt = nullptr;
  double* tpart = nullptr;
  const double** d_b = nullptr;    // the caller's vector pointers, on the device
  double** d_x = nullptr;
  void** host_ptrs = nullptr;      // pinned staging of those pointers (2 nsys)
  int grid_max = 0;                // co-resident CTAs of the most occupant variant
  int vmax[kVariants] = {};        // co-resident CTAs of each kernel variant
  int grid_tuned[4] = {};          // chosen CTAs per tune_slot (0: not yet)
  int var_tuned[4] = {};           // chosen kernel variant per tune_slot
  int tune_chosen[4] = {-1, -1, -1, -1};  // index of the chosen candidate
  float tune_ms[4][kMaxCand] = {}; // autotuner timings of the candidates
  int tune_grid[4][kMaxCand] = {};
  int tune_minb[4][kMaxCand] = {};
  int tune_count[4] = {};
  // graph of one solve: status clear, gather, init, the persistent kernel, scatter
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int gkey_jac = -1, gkey_grid = -1, gkey_var = -1, gkey_maxit = -1, gkey_restarts = -1;
  int gkey_f32 = -1, gkey_carry = -1, gkey_outer = -1;
  double gkey_tol = -1.0, gkey_timeout = -1.0, gkey_tol_in = -1.0;
  unsigned gkey_skip = 0;
  std::string graph_refused;       // why graph capture failed (then: direct launches)
  cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
  bool ran_graph = false;          // form of the last solve
  std::vector<int> host_status, host_iters, host_restarts;
  std::vector<double> host_relres;
};

void cgi::batch_free(BatchData* b) {
  if (!b) return;
  for (cg_handle* h : b->sys) cg_destroy(h);
  void* dev[] = {b->d_tstart, b->d_ntile, b->soff,     b->col,    b->d_n,  b->d_r0,   b->val[0],
                 b->val[1],   b->dg,      b->dsq,      b->disq,   b->r,    b->p,      b->q,
                 b->xh,       b->bh,      b->rho,      b->rr,     b->bb,   b->alpha,  b->beta,
                 b->relres,   b->k,       b->restarts, b->status, b->zero, b->sstate, b->cnt,
                 b->tpart,    (void*)b->d_b, (void*)b->d_x, b->d_gstart, b->d_ngroup, b->d_dmin, b->wrr, b->d_wcost,
                 b->d_sdia,   b->d_sdelta, b->val32[0], b->val32[1], b->r32, b->p32, b->q32, b->d32,
                 b->rho_k,    b->beta0,   b->stopin, b->start};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (b->host_ptrs) cudaFreeHost(b->host_ptrs);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

namespace {

cg_status bfail(cg_handle* h, cg_status s, const std::string& msg) {
  h->err = msg;
  return s;
}

#define CGB_CUDA(h, call)                                                                    \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return bfail((h), e_ == cudaErrorMemoryAllocation ? CG_ERR_OOM : CG_ERR_CUDA,          \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

// The concatenated values for one preconditioner (columns written with the first).
cg_status ensure_batch_vals(cg_handle* h, bool jac) {
  BatchData* B = h->batch;
  if (B->val[jac]) return CG_OK;
  const bool write_col = !B->val[0] && !B->val[1];
  CGB_CUDA(h, cudaMalloc(&B->val[jac], sizeof(double) * (size_t)std::max<int64_t>(B->entries, 32)));
  for (int s = 0; s < B->nsys; ++s) {
    const cg_handle* hs = B->sys[(size_t)s];
    const int64_t npad = (int64_t)B->ntile[(size_t)s] * kTile;
    const int64_t r0 = B->r0[(size_t)s];
    const int64_t sl0 = (int64_t)B->tstart[(size_t)s] * kWarps;
    int32_t* col = write_col ? B->col : nullptr;
    if (B->sdia[(size_t)s]) {
      BatchDelta bd{};
      bd.nd = B->sdia[(size_t)s];
      for (int m = 0; m < kBatchDiag; ++m) bd.d[m] = B->sdelta[(size_t)s * kBatchDiag + m];
      if (jac)
        batch_fill_dia_kernel<true><<<blocks_for(npad), 256, 0, h->stream>>>(
            hs->n, npad, sl0, hs->rowptr, hs->colind, hs->vals, B->disq + r0, B->soff, bd, B->val[jac]);
      else
        batch_fill_dia_kernel<false><<<blocks_for(npad), 256, 0, h->stream>>>(
            hs->n, npad, sl0, hs->rowptr, hs->colind, hs->vals, B->disq + r0, B->soff, bd, B->val[jac]);
      continue;
    }
    if (jac)
      batch_fill_kernel<true><<<blocks_for(npad), 256, 0, h->stream>>>(
          hs->n, npad, r0, sl0, hs->rowptr, hs->colind, hs->vals, B->disq + r0, B->soff, col, B->val[jac]);
    else
      batch_fill_kernel<false><<<blocks_for(npad), 256, 0, h->stream>>>(
          hs->n, npad, r0, sl0, hs->rowptr, hs->colind, hs->vals, B->disq + r0, B->soff, col, B->val[jac]);
  }
  CGB_CUDA(h, cudaGetLastError());
  CGB_CUDA(h, cudaStreamSynchronize(h->stream));
  return CG_OK;
}

// fp32 copies of the loop matrix, the inner vectors and the per-system inner state.
cg_status ensure_batch_f32(cg_handle* h, bool jac) {
  BatchData* B = h->batch;
  if (B->val32[jac]) return CG_OK;
  const cg_status vs = ensure_batch_vals(h, jac);
  if (vs != CG_OK) return vs;
  const size_t ent = (size_t)std::max<int64_t>(B->entries, 32);
  CGB_CUDA(h, cudaMalloc(&B->val32[jac], sizeof(float) * ent));
  batch_to_f32_kernel<<<blocks_for((int64_t)ent), 256, 0, h->stream>>>((int64_t)ent, B->val[jac], B->val32[jac]);
  CGB_CUDA(h, cudaGetLastError());
  if (!B->r32) {
    const size_t nv = (size_t)B->rows, ns = (size_t)B->nsys;
    for (float** v : {&B->r32, &B->p32, &B->q32, &B->d32}) {
      CGB_CUDA(h, cudaMalloc(v, sizeof(float) * nv));
      CGB_CUDA(h, cudaMemsetAsync(*v, 0, sizeof(float) * nv, h->stream));
    }
    for (double** v : {&B->rho_k, &B->beta0, &B->stopin}) CGB_CUDA(h, cudaMalloc(v, sizeof(double) * ns));
    CGB_CUDA(h, cudaMalloc(&B->start, sizeof(int) * ns));
  }
  CGB_CUDA(h, cudaStreamSynchronize(h->stream));
  return CG_OK;
}

BatchParams make_params(cg_handle* h, bool jac, double tol, int maxit) {
  BatchData* B = h->batch;
  BatchParams P{};
  P.nsys = B->nsys;
  P.tstart = B->d_tstart;
  P.ntile = B->d_ntile;
  P.gstart = B->d_gstart;
  P.ngroup = B->d_ngroup;
  P.wcost = B->d_wcost;
  P.sdia = B->d_sdia;
  P.sdelta = B->d_sdelta;
  P.dmin = B->d_dmin;
  P.wrr = B->wrr;
  P.soff = B->soff;
  P.col = B->col;
  P.val = B->val[jac];
  P.dg = B->dg;
  P.r = B->r;
  P.p = B->p;
  P.q = B->q;
  P.xh = B->xh;
  P.bh = B->bh;
  P.rho = B->rho;
  P.rr = B->rr;
  P.bb = B->bb;
  P.alpha = B->alpha;
  P.beta = B->beta;
  P.relres = B->relres;
  P.k = B->k;
  P.restarts = B->restarts;
  P.status = B->status;
  P.zero = B->zero;
  P.sstate = B->sstate;
  P.cnt = B->cnt;
  P.tpart = B->tpart;
  P.tol = tol;
  P.maxit = maxit;
  P.max_restarts = h->max_restarts;
  P.st = h->st;
  P.timeout_ns = (uint64_t)(h->timeout_ms * 1e6);
  P.skip_seq = h->skip_seq;
  P.val32 = B->val32[jac];
  P.r32 = B->r32;
  P.p32 = B->p32;
  P.q32 = B->q32;
  P.d32 = B->d32;
  P.rho_k = B->rho_k;
  P.beta0 = B->beta0;
  P.stopin = B->stopin;
  P.start = B->start;
  P.max_outer = h->max_outer;
  return P;
}

// The work of one solve on h->stream: clear the status words, gather b and
// x, reset the systems, the persistent kernel on G CTAs and (unless this is
// an autotuner trial, which must leave x alone) the scatter of x.
cudaError_t enqueue_solve(cg_handle* h, cudaStream_t s, bool jac, int var, int G, double tol, int maxit,
                          bool scatter, bool f32, bool carry, double tol_in) {
  BatchData* B = h->batch;
  BatchParams P = make_params(h, jac, tol, maxit);
  P.carry = carry ? 1 : 0;
  P.tol_in = tol_in;
  const dim3 gg(64, (unsigned)B->nsys);
  cudaError_t e = cudaMemsetAsync(h->st, 0, sizeof(DevState), s);
  if (e != cudaSuccess) return e;
  batch_gather_kernel<<<gg, 256, 0, s>>>(B->d_b, B->d_x, B->d_n, B->d_r0, B->d_ntile, B->disq, B->dsq,
                                          jac ? 1 : 0, B->bh, B->xh);
  batch_init_kernel<<<blocks_for(B->nsys), 256, 0, s>>>(B->nsys, B->bb, B->k, B->restarts, B->status,
                                                         B->zero, B->wrr, B->sstate, B->cnt);
  if (f32) batch_init_f32_kernel<<<blocks_for(B->nsys), 256, 0, s>>>(B->nsys, B->rho_k, B->start);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  void* args[] = {&P};
  e = cudaLaunchCooperativeKernel(batch_kernel(jac, var, f32), dim3((unsigned)G), dim3(kBlock), args, 0, s);
  if (e != cudaSuccess || !scatter) return e;
  batch_scatter_kernel<<<gg, 256, 0, s>>>(B->d_x, B->d_n, B->d_r0, B->disq, jac ? 1 : 0, B->xh, B->zero);
  return cudaGetLastError();
}

// Run one solve (through the cached graph when use_graph) between the
// handle's events; the device time goes to *ms.
cg_status run_solve(cg_handle* h, bool jac, int var, int G, double tol, int maxit, bool use_graph,
                    bool scatter, float* ms, bool f32, bool carry, double tol_in) {
  BatchData* B = h->batch;
  if (use_graph && B->graph_refused.empty()) {
    const bool same = B->gexec && B->gkey_jac == (int)jac && B->gkey_grid == G && B->gkey_var == var &&
                      B->gkey_tol == tol && B->gkey_f32 == (int)f32 && B->gkey_carry == (int)carry &&
                      B->gkey_tol_in == tol_in && B->gkey_outer == h->max_outer &&
                      B->gkey_maxit == maxit && B->gkey_restarts == h->max_restarts &&
                      B->gkey_timeout == h->timeout_ms && B->gkey_skip == h->skip_seq;
    if (!same) {
      if (B->gexec) cudaGraphExecDestroy(B->gexec);
      if (B->graph) cudaGraphDestroy(B->graph);
      B->gexec = nullptr;
      B->graph = nullptr;
      B->gkey_jac = -1;
      // captured on a private stream (the caller's may be the legacy stream, which
      // cannot capture); the graph is then launched on the caller's stream
      if (!B->cap_stream) CGB_CUDA(h, cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
      CGB_CUDA(h, cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
      const cudaError_t e = enqueue_solve(h, B->cap_stream, jac, var, G, tol, maxit, true, f32, carry, tol_in);
      cudaGraph_t graph = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(B->cap_stream, &graph);
      cudaError_t e3 = cudaSuccess;
      if (e == cudaSuccess && e2 == cudaSuccess) e3 = cudaGraphInstantiate(&B->gexec, graph, 0);
      if (e != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        // a runtime that cannot capture or instantiate the cooperative launch:
        // run the same kernels as direct launches from now on
        if (graph) cudaGraphDestroy(graph);
        B->gexec = nullptr;
        cudaGetLastError();
        B->graph_refused = cudaGetErrorString(e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : e3));
        return run_solve(h, jac, var, G, tol, maxit, false, scatter, ms, f32, carry, tol_in);
      }
      B->graph = graph;
      B->gkey_jac = jac;
      B->gkey_grid = G;
      B->gkey_var = var;
      B->gkey_tol = tol;
      B->gkey_maxit = maxit;
      B->gkey_restarts = h->max_restarts;
      B->gkey_timeout = h->timeout_ms;
      B->gkey_skip = h->skip_seq;
      B->gkey_f32 = f32;
      B->gkey_carry = carry;
      B->gkey_tol_in = tol_in;
      B->gkey_outer = h->max_outer;
    }
    CGB_CUDA(h, cudaEventRecord(h->ev0, h->stream));
    CGB_CUDA(h, cudaGraphLaunch(B->gexec, h->stream));
    CGB_CUDA(h, cudaEventRecord(h->ev1, h->stream));
    B->ran_graph = true;
  } else {
    B->ran_graph = false;
    CGB_CUDA(h, cudaEventRecord(h->ev0, h->stream));
    const cudaError_t e = enqueue_solve(h, h->stream, jac, var, G, tol, maxit, scatter, f32, carry, tol_in);
    if (e != cudaSuccess)
      return bfail(h, e == cudaErrorMemoryAllocation ? CG_ERR_OOM : CG_ERR_CUDA,
                   std::string("cg_solve_batch: launch: ") + cudaGetErrorString(e));
    CGB_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  }
  CGB_CUDA(h, cudaMemcpyAsync(h->host_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CGB_CUDA(h, cudaStreamSynchronize(h->stream));
  CGB_CUDA(h, cudaEventElapsedTime(ms, h->ev0, h->ev1));
  if (h->host_st->abort)
    return bfail(h, CG_ERR_TIMEOUT, "cg_solve_batch: grid barrier " + std::to_string(h->host_st->err_barrier) +
                                        " timed out in CTA " + std::to_string(h->host_st->err_cta));
  return CG_OK;
}

// Autotuner: the kernel variant (registers budgeted for 3, 4 or 5 CTAs per SM)
// and grid size for this handle and preconditioner, picked by timing short
// trial solves (at most kTrialIters iterations each, x left untouched) of the
// caller's own systems; the choice is kept in the handle.  Candidates: every
// variant at its full residency, and the 3-CTA variant at one CTA per SM.
constexpr int kTrialIters = 40;

cg_status autotune(cg_handle* h, bool jac, double tol, int maxit, bool f32, bool carry, double tol_in) {
  const int sl = tune_slot(jac, f32);
  BatchData* B = h->batch;
  std::vector<std::pair<int, int>> cand;  // (variant, grid)
  for (int v = 0; v < kVariants; ++v)
    if (B->vmax[v] > 0) cand.emplace_back(v, B->vmax[v]);
  if (B->vmax[0] > h->sm_count) cand.emplace_back(0, h->sm_count);
  float best = 3.0e38f;
  int best_i = 0, nt = 0;
  for (size_t c = 0; c < cand.size() && nt < kMaxCand; ++c) {
    float ms = 0.0f;
    const cg_status ts = run_solve(h, jac, cand[c].first, cand[c].second, tol,
                                   std::min<int32_t>(maxit, kTrialIters), false, false, &ms, f32, carry, tol_in);
    if (ts != CG_OK) return ts;
    B->tune_ms[sl][nt] = ms;
    B->tune_grid[sl][nt] = cand[c].second;
    B->tune_minb[sl][nt] = kVariantMinBlocks[cand[c].first];
    if (ms < best) {
      best = ms;
      best_i = nt;
    }
    ++nt;
  }
  B->tune_count[sl] = nt;
  B->tune_chosen[sl] = best_i;
  B->var_tuned[sl] = cand[(size_t)best_i].first;
  B->grid_tuned[sl] = cand[(size_t)best_i].second;
  return CG_OK;
}

}  // namespace

extern "C" {

cg_status cg_batch_create(int32_t nsys, const int64_t* n, const int32_t* const* rowptr,
                          const int32_t* const* colind, const double* const* vals, cg_handle** out) {
  if (!out) {
    cgi::set_create_error("cg_batch_create: out is NULL");
    return CG_ERR_INVALID;
  }
  *out = nullptr;
  if (nsys <= 0 || nsys > kMaxBatch) {
    cgi::set_create_error("cg_batch_create: nsys must be in [1, " + std::to_string(kMaxBatch) + "]");
    return CG_ERR_INVALID;
  }
  if (!n || !rowptr || !colind || !vals) {
    cgi::set_create_error("cg_batch_create: NULL array");
    return CG_ERR_INVALID;
  }
  for (int s = 0; s < nsys; ++s)
    if (n[s] <= 0 || n[s] >= INT32_MAX) {
      cgi::set_create_error("cg_batch_create: system " + std::to_string(s) + " has n outside [1, 2^31-1)");
      return CG_ERR_INVALID;
    }
  cg_handle* h = new cg_handle();
  BatchData* B = new BatchData();
  h->batch = B;
  auto bail = [&](cg_status s) {
    cgi::set_create_error(h->err);
    cg_destroy(h);
    return s;
  };
#define CGB_CREATE(call)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return bail(bfail(h, e_ == cudaErrorMemoryAllocation ? CG_ERR_OOM : CG_ERR_CUDA,     \
                        std::string(#call) + ": " + cudaGetErrorString(e_)));              \
  } while (0)
  int dev = 0;
  CGB_CREATE(cudaGetDevice(&dev));
  CGB_CREATE(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev));
  CGB_CREATE(cudaMalloc(&h->st, sizeof(DevState)));
  CGB_CREATE(cudaMallocHost(&h->host_st, sizeof(DevState)));
  CGB_CREATE(cudaEventCreate(&h->ev0));
  CGB_CREATE(cudaEventCreate(&h->ev1));
  B->nsys = nsys;
  B->n.assign(n, n + nsys);
  B->r0.resize((size_t)nsys);
  B->tstart.resize((size_t)nsys);
  B->ntile.resize((size_t)nsys);
  int64_t rows = 0, tiles = 0, nnz = 0;
  for (int s = 0; s < nsys; ++s) {
    cg_handle* hs = nullptr;
    const cg_status st = cg_create(n[s], rowptr[s], colind[s], vals[s], &hs);
    if (st != CG_OK)
      return bail(bfail(h, st, "cg_batch_create: system " + std::to_string(s) + ": " + cg_last_error(nullptr)));
    B->sys.push_back(hs);
    B->r0[(size_t)s] = rows;
    B->tstart[(size_t)s] = (int32_t)tiles;
    const int64_t nt = (n[s] + kTile - 1) / kTile;
    B->ntile[(size_t)s] = (int32_t)nt;
    rows += nt * kTile;
    tiles += nt;
    nnz += hs->nnz;
    if (rows >= INT32_MAX) return bail(bfail(h, CG_ERR_INVALID, "cg_batch_create: 2^31 rows or more in all"));
  }
  B->rows = rows;
  B->ntiles = (int)tiles;
  B->nslices = (int)(tiles * kWarps);
  h->n = rows;
  h->nnz = nnz;
  // layout of each system: diagonal (stencils: every off-diagonal entry on one
  // of at most kBatchDiag offsets; a slot per offset, no column array read)
  // or sliced ELL; slice widths: the offsets, or the longest off-diagonal row
  // of each 32-row slice
  B->sdia.assign((size_t)nsys, 0);
  B->sdelta.assign((size_t)nsys * kBatchDiag, 0);
  std::vector<int32_t> soff((size_t)B->nslices + 1, 0);
  int64_t off = 0;
  for (int s = 0; s < nsys; ++s) {
    cg_handle* hs = B->sys[(size_t)s];
    const cg_status so = cgi::ensure_offsets(hs);
    if (so != CG_OK) return bail(bfail(h, so, "cg_batch_create: system " + std::to_string(s) + ": " + hs->err));
    if (hs->noffs_all >= 1 && hs->noffs_all <= kBatchDiag) {
      B->sdia[(size_t)s] = hs->noffs_all;
      for (int m = 0; m < hs->noffs_all; ++m) B->sdelta[(size_t)s * kBatchDiag + m] = hs->offs_all[m];
      const int nsl = B->ntile[(size_t)s] * kWarps;
      for (int j = 0; j < nsl; ++j) {
        off += hs->noffs_all;
        soff[(size_t)B->tstart[(size_t)s] * kWarps + j + 1] = (int32_t)off;
      }
      if (off * 32 >= INT32_MAX) return bail(bfail(h, CG_ERR_INVALID, "cg_batch_create: matrices too large"));
      continue;
    }
    std::vector<int32_t> nd((size_t)hs->n);
    CGB_CREATE(cudaMemcpy(nd.data(), hs->ndiag, sizeof(int32_t) * (size_t)hs->n, cudaMemcpyDeviceToHost));
    const std::vector<int32_t>& rp = hs->host_rowptr;
    const int nsl = B->ntile[(size_t)s] * kWarps;
    for (int j = 0; j < nsl; ++j) {
      int w = 0;
      const int64_t i1 = std::min<int64_t>(hs->n, (int64_t)j * 32 + 32);
      for (int64_t i = (int64_t)j * 32; i < i1; ++i)
        w = std::max(w, rp[(size_t)i + 1] - rp[(size_t)i] - nd[(size_t)i]);
      off += w;
      soff[(size_t)B->tstart[(size_t)s] * kWarps + j + 1] = (int32_t)off;
    }
    if (off * 32 >= INT32_MAX) return bail(bfail(h, CG_ERR_INVALID, "cg_batch_create: matrices too large"));
  }
  B->entries = off * 32;
  const size_t nv = (size_t)rows, ns = (size_t)nsys;
  CGB_CREATE(cudaMalloc(&B->soff, sizeof(int32_t) * soff.size()));
  CGB_CREATE(cudaMemcpy(B->soff, soff.data(), sizeof(int32_t) * soff.size(), cudaMemcpyHostToDevice));
  const bool any_ell = std::count(B->sdia.begin(), B->sdia.end(), 0) > 0;
  CGB_CREATE(cudaMalloc(&B->col, sizeof(int32_t) * (size_t)std::max<int64_t>(any_ell ? B->entries : 0, 32)));
  CGB_CREATE(cudaMalloc(&B->d_tstart, sizeof(int32_t) * ns));
  CGB_CREATE(cudaMalloc(&B->d_ntile, sizeof(int32_t) * ns));
  CGB_CREATE(cudaMalloc(&B->d_n, sizeof(int64_t) * ns));
  CGB_CREATE(cudaMalloc(&B->d_r0, sizeof(int64_t) * ns));
  CGB_CREATE(cudaMemcpy(B->d_tstart, B->tstart.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice));
  CGB_CREATE(cudaMemcpy(B->d_ntile, B->ntile.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice));
  CGB_CREATE(cudaMemcpy(B->d_n, B->n.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice));
  CGB_CREATE(cudaMemcpy(B->d_r0, B->r0.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice));
  for (double** v : {&B->dg, &B->dsq, &B->disq, &B->r, &B->p, &B->q, &B->xh, &B->bh})
    CGB_CREATE(cudaMalloc(v, sizeof(double) * nv));
  for (double** v : {&B->rho, &B->rr, &B->bb, &B->alpha, &B->beta, &B->relres})
    CGB_CREATE(cudaMalloc(v, sizeof(double) * ns));
  for (int** v : {&B->k, &B->restarts, &B->status, &B->zero, &B->wrr}) CGB_CREATE(cudaMalloc(v, sizeof(int) * ns));
  {
    std::vector<int32_t> gst(ns), ngr(ns), wc(ns);
    std::vector<double> dmin(ns);
    int groups = 0;
    for (size_t s = 0; s < ns; ++s) {
      gst[s] = groups;
      ngr[s] = (B->ntile[s] + kGroup - 1) / kGroup;
      groups += ngr[s];
      dmin[s] = B->sys[s]->jacobi_ok ? B->sys[s]->dmin : 1.0;
      // SpMV-phase cost of a row: W + 2 units for W stored entries a row
      // (padding included).  The phase is held by GB300's fp64 pipe (W fused
      // multiply-adds, the p.q term and the reduction) about as much as by the
      // W values (and columns) it streams; both grow as W + ~1.6
      const int64_t sl0 = (int64_t)B->tstart[s] * kWarps, sl1 = sl0 + (int64_t)B->ntile[s] * kWarps;
      const int64_t wsum = soff[(size_t)sl1] - soff[(size_t)sl0];
      const int64_t wavg = (wsum + (sl1 - sl0) - 1) / std::max<int64_t>(sl1 - sl0, 1);
      wc[s] = (int32_t)(wavg + 2);
    }
    B->ngroups = groups;
    CGB_CREATE(cudaMalloc(&B->d_gstart, sizeof(int32_t) * ns));
    CGB_CREATE(cudaMalloc(&B->d_ngroup, sizeof(int32_t) * ns));
    CGB_CREATE(cudaMalloc(&B->d_dmin, sizeof(double) * ns));
    CGB_CREATE(cudaMemcpy(B->d_gstart, gst.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice));
    CGB_CREATE(cudaMemcpy(B->d_ngroup, ngr.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice));
    CGB_CREATE(cudaMemcpy(B->d_dmin, dmin.data(), sizeof(double) * ns, cudaMemcpyHostToDevice));
    CGB_CREATE(cudaMalloc(&B->d_wcost, sizeof(int32_t) * ns));
    CGB_CREATE(cudaMemcpy(B->d_wcost, wc.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice));
    CGB_CREATE(cudaMalloc(&B->d_sdia, sizeof(int32_t) * ns));
    CGB_CREATE(cudaMemcpy(B->d_sdia, B->sdia.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice));
    CGB_CREATE(cudaMalloc(&B->d_sdelta, sizeof(int32_t) * ns * kBatchDiag));
    CGB_CREATE(cudaMemcpy(B->d_sdelta, B->sdelta.data(), sizeof(int32_t) * ns * kBatchDiag,
                          cudaMemcpyHostToDevice));
  }
  CGB_CREATE(cudaMalloc(&B->sstate, sizeof(unsigned long long) * ns));
  CGB_CREATE(cudaMalloc(&B->cnt, sizeof(unsigned) * ns));
  CGB_CREATE(cudaMalloc(&B->tpart, sizeof(double) * (size_t)B->ngroups * kWarps * kNP));
  CGB_CREATE(cudaMalloc((void**)&B->d_b, sizeof(double*) * ns));
  CGB_CREATE(cudaMalloc((void**)&B->d_x, sizeof(double*) * ns));
  CGB_CREATE(cudaMallocHost((void**)&B->host_ptrs, sizeof(void*) * 2 * ns));
  for (int s = 0; s < nsys; ++s) {
    const cg_handle* hs = B->sys[(size_t)s];
    const int64_t npad = (int64_t)B->ntile[(size_t)s] * kTile;
    batch_diag_kernel<<<blocks_for(npad), 256>>>(hs->n, npad, B->r0[(size_t)s], hs->diag, B->dg, B->dsq,
                                                 B->disq);
  }
  CGB_CREATE(cudaGetLastError());
  CGB_CREATE(cudaDeviceSynchronize());
  for (int v = 0; v < kVariants; ++v) {
    int per_sm = 1 << 20;
    for (int kind = 0; kind < 4; ++kind) {
      int ps = 0;
      CGB_CREATE(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, batch_kernel(kind & 1, v, kind >= 2), kBlock, 0));
      per_sm = std::min(per_sm, ps);
    }
    B->vmax[v] = per_sm * h->sm_count;
    B->grid_max = std::max(B->grid_max, B->vmax[v]);
  }
#undef CGB_CREATE
  if (B->grid_max <= 0) return bail(bfail(h, CG_ERR_CUDA, "cg_batch_create: occupancy query failed"));
  h->grid_max = B->grid_max;
  B->host_status.assign(ns, 0);
  B->host_iters.assign(ns, 0);
  B->host_restarts.assign(ns, 0);
  B->host_relres.assign(ns, 0.0);
  *out = h;
  return CG_OK;
}

cg_status cg_solve_batch(cg_handle* h, const double* const* b, double* const* x, double tol, int32_t maxit,
                         int32_t precond, int32_t precision, int32_t* iters, double* relres) {
  if (!h) return CG_ERR_INVALID;
  BatchData* B = h->batch;
  if (!B) return bfail(h, CG_ERR_INVALID, "cg_solve_batch: not a batch handle (made by cg_create)");
  h->last = cg_solve_info{};
  if (!b || !x || !(tol >= 0.0) || maxit < 0)
    return bfail(h, CG_ERR_INVALID, "cg_solve_batch: NULL vector array, tol < 0 or maxit < 0");
  if (precond != CG_PRECOND_NONE && precond != CG_PRECOND_JACOBI)
    return bfail(h, CG_ERR_INVALID, "cg_solve_batch: unknown preconditioner");
  if (precision != CG_PREC_FP64 && precision != CG_PREC_FP32_IR && precision != CG_PREC_FP32_RU)
    return bfail(h, CG_ERR_INVALID, "cg_solve_batch: unknown precision");
  if (h->loop_mode == 3)
    return bfail(h, CG_ERR_INVALID, "cg_solve_batch: CG_OPT_LOOP_MODE 3 (unrolled) has no batch form");
  const bool jac = precond == CG_PRECOND_JACOBI;
  for (int s = 0; s < B->nsys; ++s) {
    if (!b[s] || !x[s]) return bfail(h, CG_ERR_INVALID, "cg_solve_batch: NULL vector of system " + std::to_string(s));
    if (jac && !B->sys[(size_t)s]->jacobi_ok)
      return bfail(h, CG_ERR_INVALID,
                   "cg_solve_batch: Jacobi needs a positive diagonal (system " + std::to_string(s) + ")");
  }
  const bool f32 = precision != CG_PREC_FP64;
  const bool carry = precision == CG_PREC_FP32_RU;
  const double tol_in = h->tol_in_set ? h->tol_in : (carry ? 0.1 : 1e-4);
  cg_status vs = f32 ? ensure_batch_f32(h, jac) : ensure_batch_vals(h, jac);
  if (vs != CG_OK) return vs;
  const size_t ns = (size_t)B->nsys;
  const int sl = tune_slot(jac, f32);
  // the previous solve's copies out of host_ptrs have completed (it synchronised)
  std::memcpy(B->host_ptrs, b, sizeof(void*) * ns);
  std::memcpy(B->host_ptrs + ns, x, sizeof(void*) * ns);
  CGB_CUDA(h, cudaMemcpyAsync(B->d_b, B->host_ptrs, sizeof(void*) * ns, cudaMemcpyHostToDevice, h->stream));
  CGB_CUDA(h, cudaMemcpyAsync(B->d_x, B->host_ptrs + ns, sizeof(void*) * ns, cudaMemcpyHostToDevice, h->stream));
  int G = 0, var = 0;
  if (h->grid_opt > 0) {
    // a forced grid runs on the variant with the most registers that can hold it
    G = std::min(h->grid_opt, B->grid_max);
    while (var + 1 < kVariants && B->vmax[var] < G) ++var;
  } else {
    if (B->grid_tuned[sl] == 0) {
      const cg_status ts = autotune(h, jac, tol, maxit, f32, carry, tol_in);
      if (ts != CG_OK) return ts;
    }
    G = B->grid_tuned[sl];
    var = B->var_tuned[sl];
  }
  const bool use_graph = h->loop_mode != 1;
  float ms = 0.0f;
  const cg_status rs = run_solve(h, jac, var, G, tol, maxit, use_graph, true, &ms, f32, carry, tol_in);
  if (rs != CG_OK) return rs;
  CGB_CUDA(h, cudaMemcpyAsync(B->host_iters.data(), B->k, sizeof(int) * ns, cudaMemcpyDeviceToHost, h->stream));
  CGB_CUDA(h, cudaMemcpyAsync(B->host_restarts.data(), B->restarts, sizeof(int) * ns, cudaMemcpyDeviceToHost, h->stream));
  CGB_CUDA(h, cudaMemcpyAsync(B->host_relres.data(), B->relres, sizeof(double) * ns, cudaMemcpyDeviceToHost, h->stream));
  CGB_CUDA(h, cudaMemcpyAsync(B->host_status.data(), B->status, sizeof(int) * ns, cudaMemcpyDeviceToHost, h->stream));
  CGB_CUDA(h, cudaStreamSynchronize(h->stream));
  int worst_err = 0, nconv = 0, maxk = 0, rmax = 0;
  int64_t bytes = 0;
  double relmax = 0.0;
  for (size_t s = 0; s < ns; ++s) {
    const int st = B->host_status[s], k = B->host_iters[s];
    if (iters) iters[s] = k;
    if (relres) relres[s] = B->host_relres[s];
    if (st < 0 && (worst_err == 0 || st < worst_err)) worst_err = st;
    if (st == CG_NOT_CONVERGED) ++nconv;
    maxk = std::max(maxk, k);
    rmax = std::max(rmax, B->host_restarts[s]);
    relmax = std::max(relmax, B->host_relres[s]);
    const cg_handle* hs = B->sys[s];
    // the single-system traffic model per iteration: CSR matrix and the loop's vectors
    bytes += (f32 ? 8 * hs->nnz + 4 * (hs->n + 1) + (jac ? 52 : 44) * hs->n
                  : 12 * hs->nnz + 4 * (hs->n + 1) + (jac ? 104 : 88) * hs->n) * (int64_t)k;
  }
  cg_solve_info& I = h->last;
  I.status = worst_err ? (cg_status)worst_err : (nconv ? CG_NOT_CONVERGED : CG_OK);
  I.iters = maxk;
  I.restarts = rmax;
  I.grid_ctas = G;
  I.relres_true = relmax;
  I.relres_rec = relmax;
  I.kernel_ms = ms;
  I.bytes_moved = bytes;
  I.kernel_bytes_per_iter = 0;
  I.loop_form = B->ran_graph ? 2 : 1;
  I.kernel_launches = 4;  // gather, init, the persistent kernel, scatter
  if (worst_err)
    return bfail(h, (cg_status)I.status, std::string("cg_solve_batch: at least one system ended with ") +
                                             cg_status_string(worst_err));
  return (cg_status)I.status;
}

cg_status cg_batch_get_system(const cg_handle* h, int32_t s, int32_t* status, int32_t* iters, int32_t* restarts,
                              double* relres) {
  if (!h || !h->batch || s < 0 || s >= h->batch->nsys) return CG_ERR_INVALID;
  const BatchData* B = h->batch;
  if (status) *status = B->host_status[(size_t)s];
  if (iters) *iters = B->host_iters[(size_t)s];
  if (restarts) *restarts = B->host_restarts[(size_t)s];
  if (relres) *relres = B->host_relres[(size_t)s];
  return CG_OK;
}

cg_status cg_batch_get_tuning(const cg_handle* h, int32_t precond, int32_t precision, int32_t* count,
                              int32_t* grids, int32_t* ctas_per_sm, float* ms, int32_t* chosen) {
  if (!h || !h->batch || (precond != CG_PRECOND_NONE && precond != CG_PRECOND_JACOBI)) return CG_ERR_INVALID;
  if (precision != CG_PREC_FP64 && precision != CG_PREC_FP32_IR && precision != CG_PREC_FP32_RU)
    return CG_ERR_INVALID;
  const BatchData* B = h->batch;
  const int j = tune_slot(precond == CG_PRECOND_JACOBI, precision != CG_PREC_FP64);
  if (count) *count = B->tune_count[j];
  for (int c = 0; c < B->tune_count[j]; ++c) {
    if (grids) grids[c] = B->tune_grid[j][c];
    if (ctas_per_sm) ctas_per_sm[c] = B->tune_minb[j][c];
    if (ms) ms[c] = B->tune_ms[j][c];
  }
  if (chosen) *chosen = B->tune_chosen[j];
  return CG_OK;
}

}  // extern "C"
