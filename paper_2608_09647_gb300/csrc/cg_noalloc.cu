// cg_solve_noalloc: a (Jacobi-)CG solve that allocates no memory.
//
// Some callers cannot call cudaMalloc.  Examples are a plugin or custom
// operator running inside a framework that owns all device memory through its
// own pool allocator, code that must not own device memory of its own, and a
// latency-critical loop where a cudaMalloc (which may synchronise the device)
// would stall.  For them this file provides a handle-free solve whose scratch
// memory is a fixed file-scope __device__ array.  The caller still passes the
// matrix, b and x.
//
// The scratch array holds four vectors of CG_NOALLOC_MAX_ROWS doubles (r, p,
// q, diagonal scaling) and a result block, 2 MiB in all.  Every GPU that loads
// this library holds it until the process exits.  All calls on a device share
// the one array and it keeps the last call's contents, so the kernel
// initialises everything it reads; calls that overlap on the GPU (other
// streams, other host threads) race on it and must be serialised by the caller.
//
// In host code the array's name is only a host-side stand-in: the first call
// on each device looks up its device address with cudaGetSymbolAddress (that
// device current) and passes the address to the kernel.  That first call
// should therefore come before any stream capture.
//
// One CTA runs the whole solve (no grid barrier, no co-residency needs):
// thread-per-row CSR SpMV in storage order, fixed-order block reductions, the
// same stopping rule and residual-replacement restarts as cg_solve.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/libcg.h"
#include "cg_device.cuh"

namespace {

constexpr int64_t kMaxRows = CG_NOALLOC_MAX_ROWS;
constexpr int kThreads = cg::kBlock;  // block_sum is written for this CTA size
constexpr int kMaxRestarts = 3;
constexpr int kMaxDevices = 64;

struct NoAllocResult {
  int status;
  int iters;
  int restarts;
  int pad;
  double relres;
};

// r, p, q, d (4 * kMaxRows doubles) followed by the result block.
static __device__ __align__(256) double g_noalloc_scratch[4 * kMaxRows + 8];

// One CTA.  All reads of rowptr stay within [0, n] and of colind/vals within
// [0, nnz) because the CSR is validated before it is used.
__global__ void __launch_bounds__(kThreads, 1)
    noalloc_pcg_kernel(int n, int nnz, const int32_t* __restrict__ rowptr,
                       const int32_t* __restrict__ colind, const double* __restrict__ vals,
                       const double* __restrict__ b, double* __restrict__ x, double tol,
                       int maxit, int jac, double* scratch) {
  double* r = scratch;
  double* p = r + kMaxRows;
  double* q = p + kMaxRows;
  double* d = q + kMaxRows;
  NoAllocResult* res = reinterpret_cast<NoAllocResult*>(d + kMaxRows);
  const int t = threadIdx.x;
  auto finish = [&](int status, int iters, int restarts, double relres) {
    if (t == 0) {
      res->status = status;
      res->iters = iters;
      res->restarts = restarts;
      res->relres = relres;
    }
  };

  // CSR checks: rowptr[0] = 0, rowptr[n] = nnz, non-decreasing; colind in [0, n)
  int bad = 0;
  if (t == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) bad = 1;
  for (int i = t; i < n; i += kThreads) {
    const int a = rowptr[i], e = rowptr[i + 1];
    if (a < 0 || e < a || e > nnz) bad = 1;
  }
  if (__syncthreads_or(bad)) { finish(CG_ERR_INVALID, 0, 0, 0.0); return; }
  for (int k = t; k < nnz; k += kThreads) {
    const int c = colind[k];
    if (c < 0 || c >= n) bad = 1;
  }
  if (__syncthreads_or(bad)) { finish(CG_ERR_INVALID, 0, 0, 0.0); return; }
  // Jacobi scaling d = 1/A_ii (1 without Jacobi)
  for (int i = t; i < n; i += kThreads) {
    double s = 0.0;
    bool found = false;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (colind[k] == i) { s += vals[k]; found = true; }
    if (jac && !(found && s > 0.0)) bad = 1;
    d[i] = jac ? 1.0 / s : 1.0;
  }
  if (__syncthreads_or(bad)) { finish(CG_ERR_INVALID, 0, 0, 0.0); return; }

  // (re)start: r = b - A x, p = z = d r; returns (r.z, r.r, b.b)
  auto restart = [&](double (&v)[3]) {
    v[0] = v[1] = v[2] = 0.0;
    for (int i = t; i < n; i += kThreads) {
      double s = 0.0;
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s += vals[k] * x[colind[k]];
      const double ri = b[i] - s;
      const double zi = ri * d[i];
      r[i] = ri;
      p[i] = zi;
      v[0] += ri * zi;
      v[1] += ri * ri;
      v[2] += b[i] * b[i];
    }
    cg::block_sum<3>(v);  // ends with every thread holding the sums; p is complete
  };

  double v3[3];
  restart(v3);
  const double bb = v3[2];
  if (bb == 0.0) {
    for (int i = t; i < n; i += kThreads) x[i] = 0.0;
    finish(CG_OK, 0, 0, 0.0);
    return;
  }
  const double stop = tol * sqrt(bb);
  double rho = v3[0], rr = v3[1];
  int k = 0, restarts = 0;
  for (;;) {
    int status = CG_NOT_CONVERGED;
    for (;;) {
      if (sqrt(rr) <= stop) { status = CG_OK; break; }
      if (k >= maxit) break;
      double v1[1] = {0.0};
      for (int i = t; i < n; i += kThreads) {
        double s = 0.0;
        for (int kk = rowptr[i]; kk < rowptr[i + 1]; ++kk) s += vals[kk] * p[colind[kk]];
        q[i] = s;
        v1[0] += p[i] * s;
      }
      cg::block_sum<1>(v1);
      if (!isfinite(v1[0]) || !isfinite(rho)) { status = CG_ERR_NUMERIC; break; }
      if (v1[0] <= 0.0) { status = CG_ERR_BREAKDOWN; break; }
      const double alpha = rho / v1[0];
      double v2[2] = {0.0, 0.0};
      for (int i = t; i < n; i += kThreads) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        v2[0] += ri * (ri * d[i]);
        v2[1] += ri * ri;
      }
      cg::block_sum<2>(v2);
      const double beta = v2[0] / rho;
      rho = v2[0];
      rr = v2[1];
      for (int i = t; i < n; i += kThreads) p[i] = r[i] * d[i] + beta * p[i];
      ++k;
      __syncthreads();  // p complete before the next SpMV
    }
    if (status == CG_ERR_NUMERIC || status == CG_ERR_BREAKDOWN) {
      __syncthreads();
      restart(v3);
      finish(status, k, restarts, sqrt(v3[1]) / sqrt(bb));
      return;
    }
    __syncthreads();  // x complete before the true residual
    restart(v3);      // true residual of x; also the restart state
    const double relres = sqrt(v3[1]) / sqrt(bb);
    if (!isfinite(relres)) { finish(CG_ERR_NUMERIC, k, restarts, relres); return; }
    if (relres <= tol) { finish(CG_OK, k, restarts, relres); return; }
    if (k >= maxit || restarts >= kMaxRestarts) {
      finish(CG_NOT_CONVERGED, k, restarts, relres);
      return;
    }
    ++restarts;
    rho = v3[0];
    rr = v3[1];
  }
}

std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" cg_status cg_solve_noalloc(int64_t n, int64_t nnz, const int32_t* rowptr,
                                      const int32_t* colind, const double* vals,
                                      const double* b, double* x, double tol, int32_t maxit,
                                      int32_t precond, void* cuda_stream, int32_t* iters_out,
                                      double* relres_out) {
  if (n < 0 || n > kMaxRows || nnz < 0 || nnz > INT32_MAX || !(tol >= 0.0) || maxit < 0 ||
      (precond != CG_PRECOND_NONE && precond != CG_PRECOND_JACOBI))
    return CG_ERR_INVALID;
  if (n == 0) {
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return CG_OK;
  }
  if (!rowptr || !b || !x || (nnz > 0 && (!colind || !vals))) return CG_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CG_ERR_CUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {  // once per device, with that device current
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return CG_ERR_CUDA;
      g_scratch_addr[dev] = static_cast<double*>(addr);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  noalloc_pcg_kernel<<<1, kThreads, 0, stream>>>((int)n, (int)nnz, rowptr, colind, vals, b, x, tol,
                                                 maxit, precond == CG_PRECOND_JACOBI ? 1 : 0,
                                                 scratch);
  if (cudaGetLastError() != cudaSuccess) return CG_ERR_CUDA;
  NoAllocResult hres{};
  if (cudaMemcpyAsync(&hres, scratch + 4 * kMaxRows, sizeof(hres), cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return CG_ERR_CUDA;
  if (iters_out) *iters_out = hres.iters;
  if (relres_out) *relres_out = hres.relres;
  return static_cast<cg_status>(hres.status);
}
