// Kernels of the CG hot path (one GPU, everything resident in HBM):
//   a1  CSR SpMV q = A p fused with the p.q partial sum     (Alg. 1; Sec. 3.3 fused SpMV + dot)
//   a2  alpha, x += alpha p, r -= alpha q, z = M^-1 r, r.z and r.r partials
//                                                          (Alg. 1; Sec. 3.3 fused update + r.r)
//   a3  beta, p = z + beta p                               (Alg. 1)
//   a4  convergence test on the device                     (Alg. 1, relative form)
//   a5  true residual ||b - A x|| / ||b|| in fp64         (Sec. 3.1, recomputed residual)
// The loop runs as one persistent cooperative launch: phases are separated by
// bounded grid barriers and the scalars are formed redundantly in every CTA
// from fixed-order sums of per-CTA partials, so there is no host round trip
// per iteration and results are reproducible run to run.
#pragma once

#include "cg_device.cuh"

namespace cg {

constexpr int kCap = 2048;                 // nonzeros staged per row block
constexpr int kPerThread = kCap / kBlock;  // staged nonzeros per thread

// CSR matrix view plus its row-block schedule.  Row block b covers rows
// [rb[b], rb[b+1]); it holds either <= kCap nonzeros and <= kBlock rows
// ("stream" block: products staged in shared memory, one thread per row), or
// exactly one row with more than kCap nonzeros ("long" block: the CTA strides
// over the row and reduces).
template <typename T>
struct Csr {
  int64_t n;
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ colind;
  const T* __restrict__ vals;
  const int32_t* __restrict__ rb;
  int32_t nrb;
};

// One row block of y = A x.  Returns this thread's share of sum_i w_i y_i
// (w may be null, then 0).  Stream blocks sum each row in storage order over
// rounded products, which is the oracle's order, so fp64 results match it
// bit for bit; long rows use a strided fused multiply-add and a tree.
template <typename T>
__device__ __forceinline__ double spmv_rowblock(const Csr<T>& A, const T* x, T* y, const T* w,
                                                int b, T* s_prod) {
  const int r0 = __ldg(A.rb + b), r1 = __ldg(A.rb + b + 1);
  const int k0 = __ldg(A.rowptr + r0), k1 = __ldg(A.rowptr + r1);
  const int nk = k1 - k0;
  const int t = threadIdx.x;
  double dot = 0.0;
  if (nk > kCap) {  // long row (r1 == r0 + 1 by construction)
    T acc = T(0);
    for (int k = k0 + t; k < k1; k += kBlock) acc += __ldg(A.vals + k) * x[__ldg(A.colind + k)];
    double v[1] = {(double)acc};
    block_sum<1>(v);  // fixed-order tree over the CTA
    if (t == 0) {
      const T s = (T)v[0];
      y[r0] = s;
      if (w) dot = (double)s * (double)w[r0];
    }
    return dot;
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
    if (w) dot = (double)s * (double)w[i];
  }
  __syncthreads();  // s_prod is reused by the next row block
  return dot;
}

// Stand-alone y = A x over all row blocks (cg_spmv, and setup work).
template <typename T>
__global__ void __launch_bounds__(kBlock) spmv_kernel(Csr<T> A, const T* x, T* y) {
  __shared__ T s_prod[kCap];
  for (int b = blockIdx.x; b < A.nrb; b += gridDim.x) spmv_rowblock<T>(A, x, y, nullptr, b, s_prod);
}

// ---------------------------------------------------------------------------
// Persistent solver launch
// ---------------------------------------------------------------------------

struct SolveParams {
  Csr<double> A;          // fp64 matrix
  Csr<float> A32;         // fp32 copy of the values (refinement only)
  const double* b;
  double* x;
  double *r, *p, *q;      // fp64 work vectors
  const double* dinv;     // 1 / A_ii (Jacobi)
  float *r32, *p32, *q32, *d32;
  const float* dinv32;
  double* part;           // per-CTA partials, kParts x G
  DevState* st;
  double tol;             // outer relative tolerance
  double tol_in;          // inner tolerance (refinement)
  int maxit;              // SpMV cap of the CG loop (total inner iterations for refinement)
  int max_restarts;       // residual replacements (fp64) / refinement steps (refinement)
  uint64_t timeout_ns;
  unsigned skip_seq;
};

// Partial-sum slots (each G doubles): 0 = p.q, 2/3 = r.z / r.r of the loop,
// 4..7 = the residual phase.  Disjoint slots mean a CTA never overwrites a
// partial that a slower CTA has still to read.
constexpr int kParts = 8;
constexpr int kSlotPQ = 0, kSlotRZ = 2, kSlotRes = 4;

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

// Write this CTA's block sums of v[0..NV) into part[j*G + cta].
template <int NV>
__device__ __forceinline__ void publish(double (&v)[NV], double* part, const Grid& g) {
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) part[(size_t)j * g.G + g.cta] = v[j];
  }
}

template <typename T> struct Vec;
template <> struct Vec<double> { using type = double2; static constexpr int N = 2; };
template <> struct Vec<float> { using type = float4; static constexpr int N = 4; };

template <typename T>
__device__ __forceinline__ T lane_of(const typename Vec<T>::type& v, int j);
template <> __device__ __forceinline__ double lane_of<double>(const double2& v, int j) { return j == 0 ? v.x : v.y; }
template <> __device__ __forceinline__ float lane_of<float>(const float4& v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}
template <typename T>
__device__ __forceinline__ void set_lane(typename Vec<T>::type& v, int j, T a);
template <> __device__ __forceinline__ void set_lane<double>(double2& v, int j, double a) {
  if (j == 0) v.x = a; else v.y = a;
}
template <> __device__ __forceinline__ void set_lane<float>(float4& v, int j, float a) {
  if (j == 0) v.x = a; else if (j == 1) v.y = a; else if (j == 2) v.z = a; else v.w = a;
}

// a2: x += alpha p; r -= alpha q; z = M^-1 r; partial (r.z, r.r).  16-byte
// vector loads/stores over [0, n - n % VN), scalar tail after; every vector
// starts 16-byte aligned.
template <typename T, bool JAC>
__device__ __forceinline__ void phase_update_xr(int64_t n, T* x, T* r, const T* p, const T* q,
                                                const T* dinv, T alpha, double& rz, double& rr,
                                                const Grid& g) {
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::N;
  const int64_t nv = n / VN;
  for (int64_t iv = g.gtid; iv < nv; iv += g.gstride) {
    V xv = reinterpret_cast<V*>(x)[iv];
    V rv = reinterpret_cast<V*>(r)[iv];
    const V pv = reinterpret_cast<const V*>(p)[iv];
    const V qv = reinterpret_cast<const V*>(q)[iv];
    V dv;
    if (JAC) dv = __ldg(reinterpret_cast<const V*>(dinv) + iv);
#pragma unroll
    for (int j = 0; j < VN; ++j) {
      const T xi = lane_of<T>(xv, j) + alpha * lane_of<T>(pv, j);
      const T ri = lane_of<T>(rv, j) - alpha * lane_of<T>(qv, j);
      set_lane<T>(xv, j, xi);
      set_lane<T>(rv, j, ri);
      rr += (double)ri * (double)ri;
      if (JAC) rz += (double)ri * (double)(ri * lane_of<T>(dv, j));
    }
    reinterpret_cast<V*>(x)[iv] = xv;
    reinterpret_cast<V*>(r)[iv] = rv;
  }
  for (int64_t i = nv * VN + g.gtid; i < n; i += g.gstride) {
    const T xi = x[i] + alpha * p[i];
    const T ri = r[i] - alpha * q[i];
    x[i] = xi;
    r[i] = ri;
    rr += (double)ri * (double)ri;
    if (JAC) rz += (double)ri * (double)(ri * __ldg(dinv + i));
  }
  if (!JAC) rz = rr;
}

// a3: p = z + beta p with z = M^-1 r.
template <typename T, bool JAC>
__device__ __forceinline__ void phase_update_p(int64_t n, const T* r, T* p, const T* dinv, T beta,
                                               const Grid& g) {
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::N;
  const int64_t nv = n / VN;
  for (int64_t iv = g.gtid; iv < nv; iv += g.gstride) {
    const V rv = reinterpret_cast<const V*>(r)[iv];
    V pv = reinterpret_cast<V*>(p)[iv];
    V dv;
    if (JAC) dv = __ldg(reinterpret_cast<const V*>(dinv) + iv);
#pragma unroll
    for (int j = 0; j < VN; ++j) {
      const T z = JAC ? lane_of<T>(rv, j) * lane_of<T>(dv, j) : lane_of<T>(rv, j);
      set_lane<T>(pv, j, z + beta * lane_of<T>(pv, j));
    }
    reinterpret_cast<V*>(p)[iv] = pv;
  }
  for (int64_t i = nv * VN + g.gtid; i < n; i += g.gstride) {
    const T z = JAC ? r[i] * __ldg(dinv + i) : r[i];
    p[i] = z + beta * p[i];
  }
}

// a1 over the grid: q = A p, partial p.q (row blocks dealt round-robin to CTAs).
template <typename T>
__device__ __forceinline__ double phase_spmv(const Csr<T>& A, const T* p, T* q, const Grid& g,
                                             T* s_prod) {
  double pq = 0.0;
  for (int b = (int)g.cta; b < A.nrb; b += (int)g.G) pq += spmv_rowblock<T>(A, p, q, p, b, s_prod);
  return pq;
}

// Status codes shared with the host API (values of cg_status).
constexpr int kOk = 0, kNotConverged = 1, kBreakdown = -2, kNumeric = -3, kTimeout = -4;

// The CG loop of Alg. 1 on vectors of type T starting from r, p = M^-1 r,
// rho = r.z, rr = r.r (given): iterate until sqrt(rr) <= stop_abs or maxit
// SpMVs.  Returns kOk (recursive test met), kNotConverged (maxit), kBreakdown,
// kNumeric or kTimeout; *iters is advanced by the SpMVs done; *rr_out holds
// the last r.r.
template <typename T, bool JAC>
__device__ int cg_loop(const Csr<T>& A, T* x, T* r, T* p, T* q, const T* dinv, double rho,
                       double rr, double stop_abs, int maxit, int* iters, double* rr_out,
                       double* part, Grid& g, T* s_prod) {
  int k = *iters;
  int status = kNotConverged;
  for (;;) {
    if (sqrt(rr) <= stop_abs) { status = kOk; break; }  // a4: test before the SpMV
    if (k >= maxit) break;
    {  // a1
      double v[1] = {phase_spmv<T>(A, p, q, g, s_prod)};
      publish<1>(v, part + kSlotPQ * (size_t)g.G, g);
    }
    if (!g.sync()) { status = kTimeout; break; }
    double pq[1];
    grid_sum<1>(part + kSlotPQ * (size_t)g.G, g.G, pq);
    if (!isfinite(pq[0]) || !isfinite(rho)) { status = kNumeric; break; }
    if (pq[0] <= 0.0) { status = kBreakdown; break; }
    const T alpha = (T)(rho / pq[0]);
    {  // a2
      double v[2] = {0.0, 0.0};
      phase_update_xr<T, JAC>(A.n, x, r, p, q, dinv, alpha, v[0], v[1], g);
      publish<2>(v, part + kSlotRZ * (size_t)g.G, g);
    }
    if (!g.sync()) { status = kTimeout; break; }
    double s2[2];
    grid_sum<2>(part + kSlotRZ * (size_t)g.G, g.G, s2);
    const T beta = (T)(s2[0] / rho);
    rho = s2[0];
    rr = s2[1];
    phase_update_p<T, JAC>(A.n, r, p, dinv, beta, g);  // a3
    ++k;
    if (!g.sync()) { status = kTimeout; break; }
  }
  *iters = k;
  *rr_out = rr;
  return status;
}

// a5 and (re)start: q = A x; r = b - q; z = M^-1 r; p = z; returns (r.z, r.r, b.b)
// grid sums.  Returns false on a barrier timeout.
template <bool JAC>
__device__ bool residual_phase64(const SolveParams& P, Grid& g, double* s_prod, double (&out)[3]) {
  phase_spmv<double>(P.A, P.x, P.q, g, s_prod);
  if (!g.sync()) return false;
  double v[3] = {0.0, 0.0, 0.0};
  const int64_t n = P.A.n;
  for (int64_t i = g.gtid; i < n; i += g.gstride) {
    const double bi = P.b[i];
    const double ri = bi - P.q[i];
    const double zi = JAC ? ri * __ldg(P.dinv + i) : ri;
    P.r[i] = ri;
    P.p[i] = zi;
    v[0] += ri * zi;
    v[1] += ri * ri;
    v[2] += bi * bi;
  }
  publish<3>(v, P.part + kSlotRes * (size_t)g.G, g);
  if (!g.sync()) return false;
  grid_sum<3>(P.part + kSlotRes * (size_t)g.G, g.G, out);
  return true;
}

// fp64 (Jacobi-)PCG with true-residual check and residual-replacement
// restarts (readings R1-R5 of the method; see the oracle's header).
template <bool JAC>
__global__ void __launch_bounds__(kBlock) pcg64_kernel(SolveParams P) {
  __shared__ double s_prod[kCap];
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  int status = kNotConverged, k = 0, restarts = 0;
  double relres_true = 0.0, rr = 0.0, bb = 0.0;
  bool first = true;
  for (;;) {
    double s3[3];
    if (!residual_phase64<JAC>(P, g, s_prod, s3)) { status = kTimeout; break; }
    if (first) {
      bb = s3[2];
      if (bb == 0.0) {  // b = 0: x = 0 solves it
        for (int64_t i = g.gtid; i < P.A.n; i += g.gstride) P.x[i] = 0.0;
        status = kOk;
        relres_true = 0.0;
        rr = 0.0;
        break;
      }
    } else {
      relres_true = sqrt(s3[1]) / sqrt(bb);
      if (!isfinite(relres_true)) { status = kNumeric; break; }
      if (relres_true <= P.tol) { status = kOk; break; }
      if (k >= P.maxit || restarts >= P.max_restarts) { status = kNotConverged; break; }
      ++restarts;
    }
    first = false;
    rr = s3[1];
    const int st = cg_loop<double, JAC>(P.A, P.x, P.r, P.p, P.q, P.dinv, s3[0], rr,
                                         P.tol * sqrt(bb), P.maxit, &k, &rr, P.part, g, s_prod);
    if (st == kTimeout) { status = kTimeout; break; }
    if (st == kNumeric || st == kBreakdown) {
      status = st;
      double s3e[3];
      if (residual_phase64<JAC>(P, g, s_prod, s3e)) relres_true = sqrt(s3e[1]) / sqrt(bb);
      else status = kTimeout;
      break;
    }
    // st is kOk or kNotConverged: loop back to recompute the true residual
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
// residual, solution update and convergence test, the inner fp32 Jacobi-PCG
// with fp64-accumulated dot products, all in one persistent launch.
template <bool JAC>
__global__ void __launch_bounds__(kBlock) pcg_ir_kernel(SolveParams P) {
  __shared__ double s_prod64[kCap];
  float* s_prod32 = reinterpret_cast<float*>(s_prod64);
  Grid g(P.st, P.timeout_ns, P.skip_seq);
  const int64_t n = P.A.n;
  int status = kNotConverged, inner = 0, outer = 0;
  double relres = 0.0, bb = 0.0, rr32 = 0.0;
  for (;;) {
    // outer fp64 residual r = b - A x, fused with the inner start:
    // r32 = fl32(r), d = 0, p32 = z32 = dinv32 r32
    phase_spmv<double>(P.A, P.x, P.q, g, s_prod64);
    if (!g.sync()) { status = kTimeout; break; }
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = g.gtid; i < n; i += g.gstride) {
      const double bi = P.b[i];
      const double ri = bi - P.q[i];
      const float r32 = (float)ri;
      const float z32 = JAC ? r32 * __ldg(P.dinv32 + i) : r32;
      P.r32[i] = r32;
      P.p32[i] = z32;
      P.d32[i] = 0.0f;
      v[0] += ri * ri;
      v[1] += bi * bi;
      v[2] += (double)r32 * (double)z32;
      v[3] += (double)r32 * (double)r32;
    }
    publish<4>(v, P.part + kSlotRes * (size_t)g.G, g);
    if (!g.sync()) { status = kTimeout; break; }
    double s4[4];
    grid_sum<4>(P.part + kSlotRes * (size_t)g.G, g.G, s4);
    if (outer == 0) {
      bb = s4[1];
      if (bb == 0.0) {
        for (int64_t i = g.gtid; i < n; i += g.gstride) P.x[i] = 0.0;
        status = kOk;
        relres = 0.0;
        break;
      }
    }
    relres = sqrt(s4[0]) / sqrt(bb);
    if (!isfinite(relres)) { status = kNumeric; break; }
    if (relres <= P.tol) { status = kOk; break; }
    if (outer >= P.max_restarts || inner >= P.maxit) { status = kNotConverged; break; }
    const int st = cg_loop<float, JAC>(P.A32, P.d32, P.r32, P.p32, P.q32, P.dinv32, s4[2], s4[3],
                                        P.tol_in * sqrt(s4[3]), P.maxit, &inner, &rr32, P.part, g,
                                        s_prod32);
    if (st == kTimeout || st == kNumeric || st == kBreakdown) { status = st; break; }
    // x += fl64(d); a barrier before the next SpMV reads x at neighbours
    for (int64_t i = g.gtid; i < n; i += g.gstride) P.x[i] += (double)P.d32[i];
    ++outer;
    if (!g.sync()) { status = kTimeout; break; }
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
