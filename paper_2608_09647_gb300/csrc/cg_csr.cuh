// SpMV on the caller's CSR matrix (Sec. 3.1: y_i = sum_k vals[k] x[colind[k]]
// over row i's stored entries): cg_spmv, the residuals b - A x of the graph
// form, and the once-per-solve true residual of the persistent kernels.
//
// The rows are cut on the host into row blocks of at most kCapV nonzeros and
// kBlock rows; a row with more than kCapV nonzeros is a block of its own (a
// "long" block, which the CTA strides over and reduces).  Two forms:
//
//  * spmv_rowblock_fma (the stand-alone kernel): the block's column indices and
//    values are copied to shared memory with 16-byte loads (four indices, two
//    pairs of values) starting at the 16-byte boundary at or below the block's
//    first nonzero; rows of at most 16 nonzeros are summed by one thread each
//    (storage order, fused multiply-adds: one fp64 FMA per nonzero), longer
//    rows by a warp each, and a row beyond the block cap by the whole CTA.  GB300's fp64 pipe issues 2 FMAs per clock per SM,
//    so a separate multiply and add per nonzero (two fp64 instructions) makes a
//    7-point SpMV pipe-bound; with one FMA the kernel is HBM-bound.
//  * spmv_rowblock (inside the persistent solver kernels, twice per solve):
//    products rounded, then summed in storage order, the oracle's arithmetic
//    exactly, staged in a smaller shared buffer so the persistent kernels keep
//    their occupancy.
#pragma once

#include "cg_device.cuh"

namespace cg {

constexpr int kCap = 2048;                 // shared staging of one row block (persistent kernels)
constexpr int kCapV = kCap - 4;            // nonzeros of a row block: its 16-byte window fits kCap
constexpr int kPerThread = kCap / kBlock;  // nonzeros per thread

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

// One row block of y = A x, the oracle's arithmetic: stream blocks sum each row
// in storage order over rounded products, so fp64 results match it bit for
// bit; long rows use a strided multiply-add and a fixed tree.
template <typename T>
__device__ __forceinline__ void spmv_rowblock(const Csr<T>& A, const T* x, T* y, int b, T* s_prod) {
  const int r0 = __ldg(A.rb + b), r1 = __ldg(A.rb + b + 1);
  const int k0 = __ldg(A.rowptr + r0), k1 = __ldg(A.rowptr + r1);
  const int nk = k1 - k0;
  const int t = threadIdx.x;
  if (nk > kCap) {  // long row (r1 == r0 + 1 by construction)
    T acc = T(0);
    for (int k = k0 + t; k < k1; k += kBlock) acc += __ldg(A.vals + k) * x[__ldg(A.colind + k)];
    double v[1] = {(double)acc};
    block_sum<1>(v);
    if (t == 0) y[r0] = (T)v[0];
    return;
  }
  T prod[kPerThread];
  int col[kPerThread];
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const int k = t + j * kBlock;
    if (k < nk) {
      col[j] = __ldg(A.colind + k0 + k);
      prod[j] = __ldg(A.vals + k0 + k);
    }
  }
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const int k = t + j * kBlock;
    if (k < nk) prod[j] = prod[j] * x[col[j]];
  }
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const int k = t + j * kBlock;
    if (k < nk) s_prod[k] = prod[j];
  }
  __syncthreads();
  const int i = r0 + t;
  if (i < r1) {
    const int a = __ldg(A.rowptr + i) - k0, e = __ldg(A.rowptr + i + 1) - k0;
    T s = T(0);
    for (int k = a; k < e; ++k) s += s_prod[k];
    y[i] = s;
  }
  __syncthreads();  // s_prod is reused by the next row block
}

// A row block's 16-byte window holds at most kCapV + 3 nonzeros: two quads
// (four nonzeros on a 16-byte boundary) per thread.
constexpr int kQuadPasses = 2;
static_assert((kCapV + 3 + 3) / 4 <= kQuadPasses * kBlock, "a row block's window exceeds two quads per thread");
constexpr int kRowUnroll = 4;  // a row's nonzeros whose gathers are in flight together
constexpr int kThreadRow = 16;  // rows with more nonzeros are summed by a warp each

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
    if (len > kThreadRow) {
      s_med[atomicAdd(s_nmed, 1)] = i;  // a warp sums it below (the order of the list does not matter)
      len = -1;
    }
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
