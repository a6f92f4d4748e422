// SpMV on the caller's CSR matrix (Sec. 3.1: y_i = sum_k vals[k] x[colind[k]]
// over row i's stored entries): cg_spmv, the residuals b - A x of the graph
// form, and the true residuals and refinement residuals of the persistent
// kernels.
//
// The rows are cut on the host into row blocks of at most kCapV nonzeros and
// kBlock rows; a row with more than kCapV nonzeros is a block of its own (a
// "long" block, which the CTA strides over and reduces).  spmv_rowblock_fma:
// the block's column indices and values are copied to shared memory with
// 16-byte loads (four indices, two pairs of values) starting at the 16-byte
// boundary at or below the block's first nonzero; short rows (kThreadRow)
// are summed by one thread each (storage order, fused multiply-adds: one fp64
// FMA per nonzero), longer rows by a warp each, and a row beyond the block cap
// by the whole CTA.  GB300's fp64 pipe issues 2 FMAs per clock per SM, so a
// separate multiply and add per nonzero (two fp64 instructions) makes a
// 7-point SpMV pipe-bound; with one FMA the kernel is HBM-bound.
#pragma once

#include "cg_device.cuh"

namespace cg {

constexpr int kCap = 2048;                 // shared staging of one row block
constexpr int kCapV = kCap - 4;            // nonzeros of a row block: its 16-byte window fits kCap

// CSR matrix view plus its row-block schedule.  Row block b covers rows
// [rb[b], rb[b+1]).  vec != 0: colind and vals start on 16-byte boundaries, so
// the 16-byte loads of spmv_rowblock_fma are allowed.
template <typename T>
struct Csr {
  int64_t n;
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ colind;
  const T* __restrict__ vals;
  const int32_t* __restrict__ rb;
  int32_t nrb;
  int32_t vec;
};

constexpr int kQuadPasses = 2;
static_assert((kCapV + 3 + 3) / 4 <= kQuadPasses * kBlock, "a row block's window exceeds two quads per thread");
constexpr int kRowUnroll = 4;  // a row's nonzeros whose gathers are in flight together
// Rows with more nonzeros than a thread takes are summed by a warp each.  A
// thread takes a row of up to kThreadRow entries; in the caller's CSR, when
// more than kWideRows of a warp's 32 rows have kThreadRow + 1 .. kThreadRowWide
// entries (a 27-point stencil) it takes those too: one
// thread a row costs the warp one FMA step per entry, where a warp per row adds
// a 5-level fp64 tree to every row (27 entries: ~0.84 fp64 warp instructions a
// row against ~6); a few such rows among short ones go to warps, so they do not
// hold a warp of short rows.
constexpr int kThreadRow = 16;
constexpr int kThreadRowWide = 32;
constexpr int kWideRows = 4;

// The longest row a thread of this warp keeps (all 32 lanes call it).
__device__ __forceinline__ int thread_row_limit(int len) {
  const unsigned wide = __ballot_sync(0xffffffffu, len > kThreadRow && len <= kThreadRowWide);
  return __popc(wide) > kWideRows ? kThreadRowWide : kThreadRow;
}

// One row block of y = A x with one fused multiply-add per nonzero (header
// comment).  The block's column indices and values are copied with 16-byte
// loads into s_col / s_val at their offset from the window start a0.  Rows of
// at most kThreadRow nonzeros are then summed by their own thread, in storage
// order, gathering x themselves (a warp's gathers for one term cover 32
// consecutive rows' neighbours); longer rows, listed in s_med, by a warp each
// (lanes stride over the row, a fixed xor tree joins them), so one long row
// does not hold a warp of short ones.
__device__ __forceinline__ void spmv_rowblock_fma(const Csr<double>& A, const double* __restrict__ x,
                                                  double* __restrict__ y, int b, int* s_col, double* s_val,
                                                  int* s_med, int* s_nmed) {
  const int r0 = __ldg(A.rb + b), r1 = __ldg(A.rb + b + 1);
  const int k0 = __ldg(A.rowptr + r0), k1 = __ldg(A.rowptr + r1);
  const int t = threadIdx.x;
  if (k1 - k0 > kCapV) {  // long row (r1 == r0 + 1 by construction): strided FMA, fixed tree
    double acc = 0.0;
    for (int k = k0 + t; k < k1; k += kBlock) acc = fma(__ldg(A.vals + k), __ldg(x + __ldg(A.colind + k)), acc);
    double v[1] = {acc};
    block_sum<1>(v);
    if (t == 0) y[r0] = v[0];
    return;
  }
  const int a0 = A.vec ? (k0 & ~3) : k0;
  const int nq = (k1 - a0 + 3) >> 2;
  if (t == 0) *s_nmed = 0;
  int4 c4[kQuadPasses];
  double2 va[kQuadPasses], vb[kQuadPasses];
#pragma unroll
  for (int j = 0; j < kQuadPasses; ++j) {  // every load issued before the first store
    const int qd = t + j * kBlock;
    const int k = a0 + 4 * qd;
    c4[j] = make_int4(0, 0, 0, 0);
    va[j] = vb[j] = make_double2(0.0, 0.0);
    if (qd >= nq) continue;
    if (A.vec && k + 4 <= k1) {
      c4[j] = __ldg(reinterpret_cast<const int4*>(A.colind + k));
      va[j] = __ldg(reinterpret_cast<const double2*>(A.vals + k));
      vb[j] = __ldg(reinterpret_cast<const double2*>(A.vals + k + 2));
    } else {  // the ragged end of the block (or unaligned arrays): entries below k1 only
      int c[4] = {0, 0, 0, 0};
      double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u < k1) {
          c[u] = __ldg(A.colind + k + u);
          v[u] = __ldg(A.vals + k + u);
        }
      c4[j] = make_int4(c[0], c[1], c[2], c[3]);
      va[j] = make_double2(v[0], v[1]);
      vb[j] = make_double2(v[2], v[3]);
    }
  }
#pragma unroll
  for (int j = 0; j < kQuadPasses; ++j) {
    const int qd = t + j * kBlock;
    if (qd < nq) {
      *reinterpret_cast<int4*>(s_col + 4 * qd) = c4[j];
      *reinterpret_cast<double2*>(s_val + 4 * qd) = va[j];
      *reinterpret_cast<double2*>(s_val + 4 * qd + 2) = vb[j];
    }
  }
  __syncthreads();
  const int i = r0 + t;
  int a = 0, len = 0;
  if (i < r1) {
    a = __ldg(A.rowptr + i) - a0;
    len = __ldg(A.rowptr + i + 1) - a0 - a;
  }
  if (len > thread_row_limit(len)) {
    s_med[atomicAdd(s_nmed, 1)] = i;  // a warp sums it below (the order of the list does not matter)
    len = -1;
  }
  // one row a thread; the warp's FMA chain runs to its longest row (GB300 issues
  // an fp64 warp instruction in full whatever its active lanes), each lane keeping
  // its sum past its own row's end
  const int wlen = __reduce_max_sync(0xffffffffu, len);
  if (i < r1 && len >= 0) {
    double s = 0.0;
    int k = 0;
    for (; k + kRowUnroll <= wlen; k += kRowUnroll) {  // kRowUnroll gathers in flight together
      double xv[kRowUnroll], vv[kRowUnroll];
#pragma unroll
      for (int u = 0; u < kRowUnroll; ++u) {
        const bool in = k + u < len;
        vv[u] = in ? s_val[a + k + u] : 0.0;
        xv[u] = in ? __ldg(x + s_col[a + k + u]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kRowUnroll; ++u) {
        const double nx = fma(vv[u], xv[u], s);
        s = k + u < len ? nx : s;
      }
    }
    for (; k < wlen; ++k) {
      const bool in = k < len;
      const double nx = fma(in ? s_val[a + k] : 0.0, in ? __ldg(x + s_col[a + k]) : 0.0, s);
      s = in ? nx : s;
    }
    y[i] = s;
  }
  __syncthreads();
  const int nmed = *s_nmed;
  const int lane = t & 31;
  for (int m = t >> 5; m < nmed; m += kWarps) {
    const int row = s_med[m];
    const int a = __ldg(A.rowptr + row) - a0, e = __ldg(A.rowptr + row + 1) - a0;
    double acc = 0.0;
    for (int k = a + lane; k < e; k += 32) acc = fma(s_val[k], __ldg(x + s_col[k]), acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = acc;
  }
  __syncthreads();  // s_col / s_val / s_med are reused by the next row block
}

// Stand-alone y = A x over all row blocks (cg_spmv, the graph form's residuals);
// CTAs take blocks round-robin, so the grid works on one band of rows at a time
// and the gathers of neighbouring rows meet in L2.  fp64 only.
template <typename T>
__global__ void __launch_bounds__(kBlock, 6) spmv_kernel(Csr<T> A, const T* x, T* y) {
  static_assert(sizeof(T) == sizeof(double), "the stand-alone caller-CSR SpMV is fp64");
  __shared__ __align__(16) int s_col[kCap];
  __shared__ __align__(16) double s_val[kCap];
  __shared__ int s_med[kBlock];
  __shared__ int s_nmed;
  for (int b = blockIdx.x; b < A.nrb; b += gridDim.x) spmv_rowblock_fma(A, x, y, b, s_col, s_val, s_med, &s_nmed);
}

}  // namespace cg
