// Device-side building blocks shared by the libcg kernels: bounded grid
// barrier, fixed-order block and grid reductions, vector load helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "cg_exact.cuh"

namespace cg {

constexpr int kBlock = 256;          // threads per CTA of every libcg kernel
constexpr int kWarps = kBlock / 32;

// Device status words of one persistent launch (zeroed before each launch).
struct DevState {
  unsigned long long bar_arrivals;  // grid-barrier arrivals of this launch (only grows)
  int abort;             // set by any CTA that gave up; every CTA then leaves
  int status;            // cg_status of the solve
  int iters;
  int restarts;
  int err_cta;           // CTA that first timed out (-1 none)
  int err_barrier;       // barrier sequence number where it happened
  double relres_true;
  double relres_rec;
  unsigned long long tphase[6];  // CTA 0 time (ns): SpMV, wait, r update, wait, x/p update, wait
};

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Add without a returned value, ordered after this thread's earlier writes.
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a co-resident (cooperatively launched) grid.  Every
// wait is bounded: a CTA that waits longer than timeout_ns, or sees another
// CTA's abort flag, records CG_ERR_TIMEOUT (-4) and returns false; the caller
// must then leave the kernel.  `seq` numbers the barriers of the launch
// (1-based) for the fault-injection hook: when skip_seq == seq, CTA 0 does not
// arrive, so the barrier can never complete and every CTA's wait runs out.
// With a single CTA this is a plain __syncthreads().
__device__ __forceinline__ bool grid_barrier(DevState* st, unsigned nblocks, uint64_t timeout_ns,
                                             unsigned seq, unsigned skip_seq) {
  __shared__ int s_ok;
  if (nblocks == 1) {
    __syncthreads();
    return true;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // barrier seq of this launch is complete when the arrivals reach
    // seq * nblocks: each CTA adds 1 with release order (its partials are
    // visible first) and waits for the total with acquire loads; there is no
    // last arriver to wait for and no reset
    int ok = 1;
    const unsigned long long target = (unsigned long long)seq * nblocks;
    const bool skip = (skip_seq != 0u && seq == skip_seq && blockIdx.x == 0);
    if (!skip) red_release_add_u64(&st->bar_arrivals, 1ull);
    const uint64_t t0 = global_timer_ns();
    unsigned spins = 0;
    while (ld_acquire_u64(&st->bar_arrivals) < target) {
      if (ld_relaxed_s32(&st->abort) != 0) { ok = 0; break; }
      if (((++spins) & 15u) == 0u && global_timer_ns() - t0 > timeout_ns) {
        if (atomicCAS(&st->abort, 0, 1) == 0) {
          st->err_cta = (int)blockIdx.x;
          st->err_barrier = (int)seq;
        }
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---- exact sums on the integer pipes (cg_exact.cuh).  GB300's fp64 unit issues
// one warp instruction per ~64 clocks per SM sub-partition, so a tree of fp64
// adds in one warp (5 levels for a warp, 8 for a CTA) sits on every reduction's
// critical path; these sums use integer instructions and redux.sync, and give
// the exact sum rounded once, whatever the order of the terms.

// Sum over the warp of an integer with |S| < 2^72: four limbs (three unsigned
// 22-bit ones and the signed rest), each summed by one redux.sync, recombined exactly.
__device__ __forceinline__ cg_exact::i128 warp_sum_i128(cg_exact::i128 S) {
  using cg_exact::i128;
  const unsigned l0 = (unsigned)((unsigned long long)S & 0x3FFFFFull);
  const unsigned l1 = (unsigned)((unsigned long long)(S >> 22) & 0x3FFFFFull);
  const unsigned l2 = (unsigned)((unsigned long long)(S >> 44) & 0x3FFFFFull);
  const int l3 = (int)(S >> 66);
  const unsigned s0 = __reduce_add_sync(0xffffffffu, l0);
  const unsigned s1 = __reduce_add_sync(0xffffffffu, l1);
  const unsigned s2 = __reduce_add_sync(0xffffffffu, l2);
  const int s3 = __reduce_add_sync(0xffffffffu, l3);
  return (i128)s0 + (i128)s1 * ((i128)1 << 22) + (i128)s2 * ((i128)1 << 44) + (i128)s3 * ((i128)1 << 66);
}

// warp_sum_i128 for 64-bit terms: three limbs (two unsigned 22-bit ones and the signed rest).
__device__ __forceinline__ cg_exact::i128 warp_sum64(long long X) {
  using cg_exact::i128;
  const unsigned l0 = (unsigned)((unsigned long long)X & 0x3FFFFFull);
  const unsigned l1 = (unsigned)(((unsigned long long)X >> 22) & 0x3FFFFFull);
  const int l2 = (int)(X >> 44);
  const unsigned s0 = __reduce_add_sync(0xffffffffu, l0);
  const unsigned s1 = __reduce_add_sync(0xffffffffu, l1);
  const int s2 = __reduce_add_sync(0xffffffffu, l2);
  return (i128)s0 + (i128)s1 * ((i128)1 << 22) + (i128)s2 * ((i128)1 << 44);
}

// In every lane: the exact sum of the lanes' fp64 values at the warp's scale
// (the largest exponent field among them), packed with that scale.
__device__ __forceinline__ ulonglong2 warp_exact(double v) {
  const cg_exact::Parts p = cg_exact::parts(v);
  // one redux for the scale and the NaN flag (a bad sum is NaN; any scale >= every e will do)
  const unsigned eb = __reduce_max_sync(0xffffffffu, (unsigned)p.e | (p.bad ? 0x10000u : 0u));
  const bool bad = eb > 0xFFFFu;
  const int E = bad ? 2046 : (int)(eb & 0xFFFFu);
  unsigned long long lo, hi;
  cg_exact::pack(warp_sum64(cg_exact::to_fixed(p, E)), E, bad, &lo, &hi);
  return make_ulonglong2(lo, hi);
}

// In every lane: the exact sum of the lanes' fp64 values rounded once, with no
// fp64 instruction (for loops bound by GB300's fp64 pipe, where a 5-level fp64
// xor tree would take 5 of its warp instructions).
__device__ __forceinline__ double warp_sum_exact(double v) {
  const ulonglong2 w = warp_exact(v);
  int E;
  bool bad;
  const cg_exact::i128 S = cg_exact::unpack(w.x, w.y, &E, &bad);
  return cg_exact::to_fp64_int(S, E, bad);
}

// In every lane of a warp: the packed entries held by its lanes (lanes without
// one hold zero at scale 1) moved to their largest scale and added exactly.
__device__ __forceinline__ cg_exact::i128 sum_entries(const ulonglong2& w, bool has, int* Em, bool* bad) {
  int E = 1;
  bool b = false;
  const cg_exact::i128 S = has ? cg_exact::unpack(w.x, w.y, &E, &b) : (cg_exact::i128)0;
  *Em = (int)__reduce_max_sync(0xffffffffu, (unsigned)E);
  *bad = __reduce_or_sync(0xffffffffu, b ? 1u : 0u) != 0u;
  return warp_sum_i128(cg_exact::shift_down(S, *Em - E));
}

// Sum of v over the CTA, valid in warp 0: each warp's exact sum (warp_exact),
// then warp 0 adds the 8 warp sums exactly and rounds once to fp64.  The result
// does not depend on which thread held which value.
template <int NV>
__device__ __forceinline__ void cta_sum0_exact(double (&v)[NV]) {
  __shared__ ulonglong2 s_w[NV][kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ulonglong2 w[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) w[j] = warp_exact(v[j]);
  __syncthreads();  // s_w may still be read by warp 0 of a previous call
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) s_w[j][warp] = w[j];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      int E;
      bool bad;
      const cg_exact::i128 T = sum_entries(s_w[j][lane < kWarps ? lane : 0], lane < kWarps, &E, &bad);
      v[j] = cg_exact::to_fp64(T, E, bad);
    }
  }
}

// Sum of v over the CTA in a fixed order, valid in thread 0 only.  A warp-wide
// fp64 add occupies GB300's fp64 pipe (2 lanes per clock per SM, ~64 clocks of
// one sub-partition's unit) whatever its active lanes, so the tree is kept to
// one warp: every thread stores its values,
// lane l of warp 0 sums threads l, l+32, ... in that order and the 32 lane
// sums meet in an xor-tree: 416 fp64 lane operations per value, against
// 3,328 for an xor-tree in every warp followed by every thread summing the
// warp sums (block_sum).
template <int NV>
__device__ __forceinline__ void cta_sum0_fp64(double (&v)[NV]) {
  __shared__ double s_v[NV][kBlock];
  __syncthreads();  // s_v may still be read by warp 0 of a previous call
#pragma unroll
  for (int j = 0; j < NV; ++j) s_v[j][threadIdx.x] = v[j];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double t = s_v[j][lane];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) t += s_v[j][w * 32 + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      v[j] = t;
    }
  }
}


// The CTA sum used by the loops: exact (cta_sum0_exact) or, in the fp64 persistent
// kernels, whose 128-register budget has no room for the 128-bit integer steps,
// the one-warp fp64 tree (cta_sum0_fp64).  Valid in warp 0.
template <int NV, bool EXACT = true>
__device__ __forceinline__ void cta_sum0(double (&v)[NV]) {
  if constexpr (EXACT) cta_sum0_exact<NV>(v);
  else cta_sum0_fp64<NV>(v);
}

// Sum of v over the CTA in a fixed order (warp xor-tree, then warp 0 over the
// per-warp sums); the result is returned to every thread.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double s_red[NV][kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  }
  __syncthreads();  // s_red may still be read from a previous call
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) s_red[j][warp] = v[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += s_red[j][w];
    v[j] = t;
  }
}

// The stopping test sqrt(rr) <= stop with the square root (a ~700-clock chain
// on GB300's fp64 pipe) taken only near the band.  stop2_hi = stop^2 (1 + 1e-12)
// rounded exceeds stop^2, and rr above it has sqrt(rr) above stop by ~5e-13
// relative (thousands of ulps), so the test is false without the root and the
// decision is the one sqrt(rr) <= stop gives.  A stop whose square under- or
// overflows (or NaN) gets stop2_hi = inf: always the exact test.
__device__ __forceinline__ double stop2_high(double stop) {
  const double s = stop * stop * (1.0 + 1e-12);
  return s >= 1e-300 ? s : INFINITY;
}
// The root stays inside its branch through a register dependence on an empty
// asm: the compiler had been computing it on every call.
__device__ __forceinline__ bool below_stop(double rr, double stop, double stop2_hi) {
  if (!(rr <= stop2_hi)) return false;
  double r = rr;
  asm volatile("" : "+d"(r));
  return sqrt(r) <= stop;
}

// Sum of the G per-CTA partials part[j*G + c], exact and rounded once, given to
// every thread.  Lane l of warp 0 takes partials l, l + 32, ..., kGridBatch loads
// in flight at a time, and adds them exactly at a running scale (the largest
// exponent seen: a larger one shifts the lane's sum down first); the 32 lane sums
// meet at the largest scale (sum_entries' alignment, one redux.sync a limb).
// Every CTA computes the identical value (same loads, same order), so decisions
// made from it agree across the grid without another barrier.
template <int NV>
__device__ __forceinline__ void grid_sum_exact_lanes(const double* part, unsigned G, double (&out)[NV]) {
  constexpr int kGridBatch = NV <= 2 ? 8 : 1;  // NV > 2: the once-per-solve residual sums
  __shared__ double s_out[NV];
  if (threadIdx.x < 32) {
    const unsigned lane = threadIdx.x;
    cg_exact::i128 acc[NV];
    int Ea[NV];
    bool bad[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      acc[j] = 0;
      Ea[j] = 1;
      bad[j] = false;
    }
    for (unsigned c0 = lane; c0 < G; c0 += 32u * kGridBatch) {
      double v[kGridBatch][NV];
#pragma unroll
      for (int u = 0; u < kGridBatch; ++u) {
        const unsigned c = c0 + 32u * u;
#pragma unroll
        for (int j = 0; j < NV; ++j) v[u][j] = c < G ? __ldcg(part + (size_t)j * G + c) : 0.0;
      }
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        // the batch's largest exponent field from the bits, then one value at a
        // time (few registers live: the persistent kernels are register-budgeted)
        int Eb = Ea[j];
#pragma unroll
        for (int u = 0; u < kGridBatch; ++u) {
          const int f = (int)((cg_exact::bits_of(v[u][j]) >> 52) & 0x7FF);
          bad[j] = bad[j] || f == 0x7FF;
          Eb = max(Eb, f == 0x7FF ? 1 : max(f, 1));
        }
        if (Eb > Ea[j]) {
          acc[j] = cg_exact::shift_down(acc[j], Eb - Ea[j]);
          Ea[j] = Eb;
        }
#pragma unroll
        for (int u = 0; u < kGridBatch; ++u) acc[j] += (cg_exact::i128)cg_exact::to_fixed(cg_exact::parts(v[u][j]), Eb);
      }
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      unsigned long long lo, hi;
      cg_exact::pack(acc[j], Ea[j], bad[j], &lo, &hi);
      int E;
      bool bd;
      const cg_exact::i128 T = sum_entries(make_ulonglong2(lo, hi), true, &E, &bd);
      const double r = cg_exact::to_fp64(T, E, bd);
      if (lane == 0) s_out[j] = r;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = s_out[j];
  __syncthreads();
}

// Sum of the G per-CTA partials part[j*G + c] in a fixed order (lane l of
// warp 0 adds c = l, l + 32, ... in order, then an xor tree), given to every
// thread.  Every CTA computes the identical value (same loads, same order), so
// decisions made from it agree across the grid without another barrier.  Each
// lane's loads go out kGridBatch at a time, so the sum waits for about
// G / (32 kGridBatch) L2 round trips instead of G / 32.
template <int NV>
__device__ __forceinline__ void grid_sum_fp64(const double* part, unsigned G, double (&out)[NV]) {
  constexpr int kGridBatch = NV <= 2 ? 8 : 1;  // NV > 2: the once-per-solve residual sums
  __shared__ double s_out[NV];
  if (threadIdx.x < 32) {
    const unsigned lane = threadIdx.x;
    double t[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) t[j] = 0.0;
    for (unsigned c0 = lane; c0 < G; c0 += 32u * kGridBatch) {
      double v[kGridBatch][NV];
#pragma unroll
      for (int u = 0; u < kGridBatch; ++u) {
        const unsigned c = c0 + 32u * u;
#pragma unroll
        for (int j = 0; j < NV; ++j) v[u][j] = c < G ? __ldcg(part + (size_t)j * G + c) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kGridBatch; ++u) {
        if (c0 + 32u * u < G) {
#pragma unroll
          for (int j = 0; j < NV; ++j) t[j] += v[u][j];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t[j] += __shfl_xor_sync(0xffffffffu, t[j], o);
      if (lane == 0) s_out[j] = t[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = s_out[j];
  __syncthreads();
}


// The same sum with every thread loading: thread t takes partials t, t + 256, ...
// (at most kPer = 4 of them, all loads in flight: one L2 round trip), each warp
// sums each of its kPer loads exactly (warp_exact), and warp 0 adds the warps'
// entries, one a lane, exactly and rounds once.  For G > 1024, or in the
// one-warp scalar kernels of the graph forms, the lane form.
template <int NV>
__device__ __forceinline__ void grid_sum_exact(const double* part, unsigned G, double (&out)[NV]) {
  constexpr int kPer = 4;
  if (G > (unsigned)(kPer * kBlock) || blockDim.x != (unsigned)kBlock) {
    grid_sum_exact_lanes<NV>(part, G, out);
    return;
  }
  __shared__ ulonglong2 s_w[NV][kPer * kWarps];
  __shared__ double s_out[NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int per = (int)((G + kBlock - 1) / kBlock);  // loads a thread makes (uniform)
  double v[kPer][NV];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const unsigned c = threadIdx.x + (unsigned)(k * kBlock);
#pragma unroll
    for (int j = 0; j < NV; ++j) v[k][j] = (k < per && c < G) ? __ldcg(part + (size_t)j * G + c) : 0.0;
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (k < per) {
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const ulonglong2 w = warp_exact(v[k][j]);
        if (lane == 0) s_w[j][k * kWarps + warp] = w;
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    const int ne = per * kWarps;  // <= 32 entries: one a lane
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      int E;
      bool bad;
      const cg_exact::i128 T = sum_entries(s_w[j][lane < ne ? lane : 0], lane < ne, &E, &bad);
      const double r = cg_exact::to_fp64(T, E, bad);
      if (lane == 0) s_out[j] = r;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = s_out[j];
  __syncthreads();
}

// The sum of the G per-CTA partials used by the loops: exact, or the fp64 form in
// the fp64 persistent kernels (see cta_sum0).
template <int NV, bool EXACT = true>
__device__ __forceinline__ void grid_sum(const double* part, unsigned G, double (&out)[NV]) {
  if constexpr (EXACT) grid_sum_exact<NV>(part, G, out);
  else grid_sum_fp64<NV>(part, G, out);
}

}  // namespace cg
