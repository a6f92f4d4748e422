// Device-side building blocks shared by the libcg kernels: bounded grid
// barrier, fixed-order block and grid reductions, vector load helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

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

// Sum of v over the CTA in a fixed order, valid in thread 0 only.  A warp-wide
// fp64 add occupies GB300's fp64 pipe (2 lanes per clock per SM) for 16
// clocks, so the tree is kept to one warp: every thread stores its values,
// lane l of warp 0 sums threads l, l+32, ... in that order and the 32 lane
// sums meet in an xor-tree: 416 fp64 lane operations per value, against
// 3,328 for an xor-tree in every warp followed by every thread summing the
// warp sums (block_sum).
template <int NV>
__device__ __forceinline__ void cta_sum0(double (&v)[NV]) {
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
__device__ __forceinline__ bool below_stop(double rr, double stop, double stop2_hi) {
  return rr <= stop2_hi && sqrt(rr) <= stop;
}

// Sum of the G per-CTA partials part[j*G + c] in a fixed order (lane l of
// warp 0 adds c = l, l + 32, ... in order, then an xor tree), given to every
// thread.  Every CTA computes the identical value (same loads, same order), so
// decisions made from it agree across the grid without another barrier.  Each
// lane's loads go out kGridBatch at a time, so the sum waits for about
// G / (32 kGridBatch) L2 round trips instead of G / 32.
template <int NV>
__device__ __forceinline__ void grid_sum(const double* part, unsigned G, double (&out)[NV]) {
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

}  // namespace cg
