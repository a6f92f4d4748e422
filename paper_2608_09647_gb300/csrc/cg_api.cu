// Host side of libcg: the C ABI declared in include/libcg.h.  It validates the
// CSR, cuts it into row blocks, owns the device workspace and launches the
// persistent solver kernels (cooperative launch: all CTAs co-resident, which
// the bounded grid barriers require).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/libcg.h"
#include "cg_kernels.cuh"

using namespace cg;

namespace {

thread_local std::string g_create_error;

// Device checks of a CSR whose rowptr the host has already validated:
// colind in [0, n); diagonal sum per row -> dinv (0 marks a row without a
// positive diagonal).
__global__ void validate_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ colind, const double* __restrict__ vals,
                                double* dinv, unsigned long long* counters) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int a = rowptr[i], e = rowptr[i + 1];
    double d = 0.0;
    bool found = false;
    unsigned long long bad = 0;
    for (int k = a; k < e; ++k) {
      const int c = colind[k];
      if (c < 0 || (int64_t)c >= n) { ++bad; continue; }
      if ((int64_t)c == i) { d += vals[k]; found = true; }
    }
    if (bad) atomicAdd(&counters[0], bad);
    if (found && d > 0.0) {
      dinv[i] = 1.0 / d;
    } else {
      dinv[i] = 0.0;
      atomicAdd(&counters[1], 1ull);
    }
  }
}

__global__ void to_float_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

}  // namespace

struct cg_handle {
  int64_t n = 0, nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* colind = nullptr;
  const double* vals = nullptr;
  int32_t* rb = nullptr;       // row-block boundaries [nrb + 1]
  int32_t nrb = 0;
  int64_t long_rows = 0;
  double* dinv = nullptr;
  bool jacobi_ok = false;
  float* vals32 = nullptr;     // refinement: fp32 values and work vectors (lazy)
  float* dinv32 = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
  double *r = nullptr, *p = nullptr, *q = nullptr;
  double* part = nullptr;
  DevState* st = nullptr;
  DevState* host_st = nullptr; // pinned
  double *stage_b = nullptr, *stage_x = nullptr;  // device staging of cg_solve_host (lazy)
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int sm_count = 0;
  int grid_max = 0;            // co-resident CTAs of the persistent kernels
  int grid_opt = 0;            // CG_OPT_GRID_CTAS (0 = auto)
  int max_restarts = 3;
  double timeout_ms = 2000.0;
  double tol_in = 1e-4;
  int max_outer = 30;
  unsigned skip_seq = 0;
  cg_solve_info last{};
  std::string err;
};

namespace {

cg_status fail(cg_handle* h, cg_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return s;
}

cg_status cuda_fail(cg_handle* h, cudaError_t e, const char* where) {
  return fail(h, e == cudaErrorMemoryAllocation ? CG_ERR_OOM : CG_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CG_CUDA(h, call)                                        \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Cut rows into row blocks: greedily extend a block while it stays within
// kCap nonzeros and kBlock rows; a row longer than kCap gets a block alone.
std::vector<int32_t> build_row_blocks(const std::vector<int32_t>& rowptr, int64_t n,
                                      int64_t* long_rows) {
  std::vector<int32_t> rb;
  rb.reserve((size_t)(n / 64 + 2));
  rb.push_back(0);
  int64_t r = 0, longs = 0;
  while (r < n) {
    const int64_t start = r;
    const int64_t len0 = rowptr[r + 1] - rowptr[r];
    if (len0 > kCap) {
      ++r;
      ++longs;
    } else {
      int64_t nk = 0;
      while (r < n && r - start < kBlock) {
        const int64_t len = rowptr[r + 1] - rowptr[r];
        if (nk + len > kCap) break;
        nk += len;
        ++r;
      }
    }
    rb.push_back((int32_t)r);
  }
  *long_rows = longs;
  return rb;
}

template <typename K>
int max_coresident(K kernel, int sm_count) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess)
    return 0;
  return per_sm * sm_count;
}

int auto_grid(const cg_handle* h) {
  if (h->grid_opt > 0) return std::min(h->grid_opt, h->grid_max);
  // enough CTAs for the larger of the row-block and vector work, capped by residency
  const int64_t vec_ctas = (h->n / 2 + kBlock - 1) / kBlock;
  const int64_t want = std::max<int64_t>(1, std::max<int64_t>(h->nrb, vec_ctas));
  return (int)std::min<int64_t>(want, h->grid_max);
}

cg_status ensure_fp32(cg_handle* h) {
  if (h->vals32) return CG_OK;
  const size_t nv = (size_t)std::max<int64_t>(h->n, 1);
  CG_CUDA(h, cudaMalloc(&h->vals32, sizeof(float) * (size_t)std::max<int64_t>(h->nnz, 1)));
  CG_CUDA(h, cudaMalloc(&h->dinv32, sizeof(float) * nv));
  CG_CUDA(h, cudaMalloc(&h->r32, sizeof(float) * nv));
  CG_CUDA(h, cudaMalloc(&h->p32, sizeof(float) * nv));
  CG_CUDA(h, cudaMalloc(&h->q32, sizeof(float) * nv));
  CG_CUDA(h, cudaMalloc(&h->d32, sizeof(float) * nv));
  if (h->nnz > 0)
    to_float_kernel<<<std::min<int64_t>((h->nnz + 255) / 256, 4096), 256, 0, h->stream>>>(
        h->nnz, h->vals, h->vals32);
  if (h->n > 0)
    to_float_kernel<<<std::min<int64_t>((h->n + 255) / 256, 4096), 256, 0, h->stream>>>(
        h->n, h->dinv, h->dinv32);
  CG_CUDA(h, cudaGetLastError());
  return CG_OK;
}

void free_all(cg_handle* h) {
  void* dev[] = {h->rb, h->dinv, h->vals32, h->dinv32, h->r32,  h->p32,    h->q32, h->d32,
                 h->r,  h->p,    h->q,      h->part,   h->st,   h->stage_b, h->stage_x};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (h->host_st) cudaFreeHost(h->host_st);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
}

}  // namespace

extern "C" {

const char* cg_status_string(int32_t s) {
  switch (s) {
    case CG_OK: return "CG_OK";
    case CG_NOT_CONVERGED: return "CG_NOT_CONVERGED";
    case CG_ERR_INVALID: return "CG_ERR_INVALID";
    case CG_ERR_BREAKDOWN: return "CG_ERR_BREAKDOWN";
    case CG_ERR_NUMERIC: return "CG_ERR_NUMERIC";
    case CG_ERR_TIMEOUT: return "CG_ERR_TIMEOUT";
    case CG_ERR_CUDA: return "CG_ERR_CUDA";
    case CG_ERR_OOM: return "CG_ERR_OOM";
    default: return "CG_UNKNOWN_STATUS";
  }
}

const char* cg_last_error(const cg_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

cg_status cg_create(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
                    cg_handle** out) {
  if (!out) return fail(nullptr, CG_ERR_INVALID, "cg_create: out is NULL");
  *out = nullptr;
  if (n < 0 || n >= INT32_MAX) return fail(nullptr, CG_ERR_INVALID, "cg_create: n out of range");
  if (!rowptr) return fail(nullptr, CG_ERR_INVALID, "cg_create: rowptr is NULL");
  cg_handle* h = new cg_handle();
  auto bail = [&](cg_status s) {
    g_create_error = h->err;
    free_all(h);
    delete h;
    return s;
  };
  h->n = n;
  h->rowptr = rowptr;
  h->colind = colind;
  h->vals = vals;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "cg_create: device query"));

  // rowptr checks on the host (the row-block cut needs it there anyway)
  std::vector<int32_t> hrp((size_t)n + 1);
  e = cudaMemcpy(hrp.data(), rowptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "cg_create: rowptr copy"));
  if (hrp[0] != 0) return bail(fail(h, CG_ERR_INVALID, "cg_create: rowptr[0] != 0"));
  for (int64_t i = 0; i < n; ++i)
    if (hrp[i + 1] < hrp[i]) return bail(fail(h, CG_ERR_INVALID, "cg_create: rowptr decreases at row " + std::to_string(i)));
  h->nnz = hrp[n];
  if (h->nnz > 0 && (!colind || !vals))
    return bail(fail(h, CG_ERR_INVALID, "cg_create: colind/vals NULL with nnz > 0"));

  std::vector<int32_t> rb = build_row_blocks(hrp, n, &h->long_rows);
  h->nrb = (int32_t)(rb.size() - 1);
  const size_t nv = (size_t)std::max<int64_t>(n, 1);
  e = cudaMalloc(&h->rb, sizeof(int32_t) * rb.size());
  if (e == cudaSuccess) e = cudaMemcpy(h->rb, rb.data(), sizeof(int32_t) * rb.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->dinv, sizeof(double) * nv);
  if (e == cudaSuccess) e = cudaMalloc(&h->r, sizeof(double) * nv);
  if (e == cudaSuccess) e = cudaMalloc(&h->p, sizeof(double) * nv);
  if (e == cudaSuccess) e = cudaMalloc(&h->q, sizeof(double) * nv);
  if (e == cudaSuccess) e = cudaMalloc(&h->st, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMallocHost(&h->host_st, sizeof(DevState));
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "cg_create: allocation"));

  // colind range and diagonal (device pass)
  unsigned long long* cnt = nullptr;
  e = cudaMalloc(&cnt, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(cnt, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess && n > 0) {
    validate_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 65535), 256>>>(n, rowptr, colind, vals, h->dinv, cnt);
    e = cudaGetLastError();
  }
  unsigned long long hc[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost);
  if (cnt) cudaFree(cnt);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "cg_create: validation"));
  if (hc[0] != 0)
    return bail(fail(h, CG_ERR_INVALID, "cg_create: " + std::to_string(hc[0]) + " column indices outside [0, n)"));
  h->jacobi_ok = (hc[1] == 0);

  // persistent-kernel residency (the smallest over the kernels we may launch)
  int g1 = max_coresident(pcg64_kernel<true>, h->sm_count);
  int g2 = max_coresident(pcg64_kernel<false>, h->sm_count);
  int g3 = max_coresident(pcg_ir_kernel<true>, h->sm_count);
  int g4 = max_coresident(pcg_ir_kernel<false>, h->sm_count);
  h->grid_max = std::min(std::min(g1, g2), std::min(g3, g4));
  if (h->grid_max <= 0) return bail(fail(h, CG_ERR_CUDA, "cg_create: occupancy query failed"));
  e = cudaMalloc(&h->part, sizeof(double) * (size_t)kParts * (size_t)h->grid_max);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "cg_create: partials"));
  *out = h;
  return CG_OK;
}

cg_status cg_set_stream(cg_handle* h, void* stream) {
  if (!h) return CG_ERR_INVALID;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return CG_OK;
}

cg_status cg_set_option(cg_handle* h, int32_t option, double value) {
  if (!h) return CG_ERR_INVALID;
  switch (option) {
    case CG_OPT_MAX_RESTARTS:
      if (!(value >= 0 && value <= 1000)) break;
      h->max_restarts = (int)value;
      return CG_OK;
    case CG_OPT_BARRIER_TIMEOUT_MS:
      if (!(value > 0 && value <= 600000)) break;
      h->timeout_ms = value;
      return CG_OK;
    case CG_OPT_GRID_CTAS:
      if (!(value >= 0 && value <= h->grid_max)) break;
      h->grid_opt = (int)value;
      return CG_OK;
    case CG_OPT_IR_TOL_INNER:
      if (!(value > 0 && value < 1)) break;
      h->tol_in = value;
      return CG_OK;
    case CG_OPT_IR_MAX_OUTER:
      if (!(value >= 0 && value <= 1000)) break;
      h->max_outer = (int)value;
      return CG_OK;
    case CG_OPT_DEBUG_SKIP_ARRIVAL:
      if (!(value >= 0 && value < 4e9)) break;
      h->skip_seq = (unsigned)value;
      return CG_OK;
    default:
      break;
  }
  return fail(h, CG_ERR_INVALID, "cg_set_option: bad option or value");
}

cg_status cg_spmv(cg_handle* h, const double* x, double* y) {
  if (!h) return CG_ERR_INVALID;
  if (h->n == 0) return CG_OK;
  if (!x || !y || x == y) return fail(h, CG_ERR_INVALID, "cg_spmv: x/y NULL or aliased");
  Csr<double> A{h->n, h->rowptr, h->colind, h->vals, h->rb, h->nrb};
  const unsigned grid = (unsigned)std::min<int64_t>(h->nrb, (int64_t)h->sm_count * 64);
  spmv_kernel<double><<<grid, kBlock, 0, h->stream>>>(A, x, y);
  CG_CUDA(h, cudaGetLastError());
  return CG_OK;
}

cg_status cg_solve(cg_handle* h, const double* b, double* x, double tol, int32_t maxit,
                   int32_t precond, int32_t precision, int32_t* iters_out, double* relres_out) {
  if (!h) return CG_ERR_INVALID;
  h->last = cg_solve_info{};
  if (!(tol >= 0.0) || maxit < 0) return fail(h, CG_ERR_INVALID, "cg_solve: tol < 0 or maxit < 0");
  if (precond != CG_PRECOND_NONE && precond != CG_PRECOND_JACOBI)
    return fail(h, CG_ERR_INVALID, "cg_solve: unknown preconditioner");
  if (precision != CG_PREC_FP64 && precision != CG_PREC_FP32_IR)
    return fail(h, CG_ERR_INVALID, "cg_solve: unknown precision");
  if (precond == CG_PRECOND_JACOBI && !h->jacobi_ok)
    return fail(h, CG_ERR_INVALID, "cg_solve: Jacobi needs a positive diagonal in every row");
  if (h->n == 0) {
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return CG_OK;
  }
  if (!b || !x) return fail(h, CG_ERR_INVALID, "cg_solve: b or x is NULL");
  if (!aligned16(b) || !aligned16(x)) return fail(h, CG_ERR_INVALID, "cg_solve: b and x must be 16-byte aligned");
  if (b == x) return fail(h, CG_ERR_INVALID, "cg_solve: b and x alias");
  if (precision == CG_PREC_FP32_IR) {
    cg_status s = ensure_fp32(h);
    if (s != CG_OK) return s;
  }
  const int G = auto_grid(h);
  SolveParams P{};
  P.A = Csr<double>{h->n, h->rowptr, h->colind, h->vals, h->rb, h->nrb};
  P.A32 = Csr<float>{h->n, h->rowptr, h->colind, h->vals32, h->rb, h->nrb};
  P.b = b;
  P.x = x;
  P.r = h->r;
  P.p = h->p;
  P.q = h->q;
  P.dinv = h->dinv;
  P.r32 = h->r32;
  P.p32 = h->p32;
  P.q32 = h->q32;
  P.d32 = h->d32;
  P.dinv32 = h->dinv32;
  P.part = h->part;
  P.st = h->st;
  P.tol = tol;
  P.tol_in = h->tol_in;
  P.maxit = maxit;
  P.max_restarts = precision == CG_PREC_FP64 ? h->max_restarts : h->max_outer;
  P.timeout_ns = (uint64_t)(h->timeout_ms * 1e6);
  P.skip_seq = h->skip_seq;
  void* args[] = {&P};
  const void* fn;
  if (precision == CG_PREC_FP64)
    fn = precond == CG_PRECOND_JACOBI ? (const void*)pcg64_kernel<true> : (const void*)pcg64_kernel<false>;
  else
    fn = precond == CG_PRECOND_JACOBI ? (const void*)pcg_ir_kernel<true> : (const void*)pcg_ir_kernel<false>;
  CG_CUDA(h, cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream));
  CG_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  CG_CUDA(h, cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kBlock), args, 0, h->stream));
  CG_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  CG_CUDA(h, cudaMemcpyAsync(h->host_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CG_CUDA(h, cudaStreamSynchronize(h->stream));
  float ms = 0.0f;
  CG_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  const DevState& s = *h->host_st;
  cg_status status = s.abort ? CG_ERR_TIMEOUT : (cg_status)s.status;
  h->last.status = status;
  h->last.iters = s.iters;
  h->last.restarts = s.restarts;
  h->last.grid_ctas = G;
  h->last.relres_true = s.relres_true;
  h->last.relres_rec = s.relres_rec;
  h->last.kernel_ms = ms;
  // modelled bytes of the CG loop (Sec. 3.3 phases): matrix + the vector streams
  const int64_t n = h->n, nnz = h->nnz;
  const int64_t per_iter = precision == CG_PREC_FP64
      ? 12 * nnz + 4 * (n + 1) + (precond == CG_PRECOND_JACOBI ? 104 : 88) * n
      : 8 * nnz + 4 * (n + 1) + (precond == CG_PRECOND_JACOBI ? 52 : 44) * n;
  h->last.bytes_moved = per_iter * (int64_t)s.iters;
  if (iters_out) *iters_out = s.iters;
  if (relres_out) *relres_out = s.relres_true;
  if (status == CG_ERR_TIMEOUT)
    return fail(h, status, "cg_solve: grid barrier " + std::to_string(s.err_barrier) +
                               " timed out in CTA " + std::to_string(s.err_cta));
  if (status < 0) return fail(h, status, std::string("cg_solve: ") + cg_status_string(status));
  return status;
}

cg_status cg_solve_host(cg_handle* h, const double* b_host, double* x_host, double tol,
                        int32_t maxit, int32_t precond, int32_t precision, int32_t* iters_out,
                        double* relres_out) {
  if (!h) return CG_ERR_INVALID;
  if (h->n == 0) return cg_solve(h, nullptr, nullptr, tol, maxit, precond, precision, iters_out, relres_out);
  if (!b_host || !x_host) return fail(h, CG_ERR_INVALID, "cg_solve_host: NULL buffer");
  const size_t bytes = sizeof(double) * (size_t)h->n;
  if (!h->stage_b) {
    CG_CUDA(h, cudaMalloc(&h->stage_b, bytes));
    CG_CUDA(h, cudaMalloc(&h->stage_x, bytes));
  }
  CG_CUDA(h, cudaMemcpyAsync(h->stage_b, b_host, bytes, cudaMemcpyHostToDevice, h->stream));
  CG_CUDA(h, cudaMemcpyAsync(h->stage_x, x_host, bytes, cudaMemcpyHostToDevice, h->stream));
  cg_status s = cg_solve(h, h->stage_b, h->stage_x, tol, maxit, precond, precision, iters_out, relres_out);
  if (s >= 0 || s == CG_ERR_BREAKDOWN || s == CG_ERR_NUMERIC) {
    CG_CUDA(h, cudaMemcpyAsync(x_host, h->stage_x, bytes, cudaMemcpyDeviceToHost, h->stream));
    CG_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return s;
}

cg_status cg_get_solve_info(const cg_handle* h, cg_solve_info* out) {
  if (!h || !out) return CG_ERR_INVALID;
  *out = h->last;
  return CG_OK;
}

cg_status cg_get_matrix_info(const cg_handle* h, int64_t* n, int64_t* nnz, int64_t* row_blocks,
                             int64_t* long_rows, int32_t* grid_ctas) {
  if (!h) return CG_ERR_INVALID;
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (row_blocks) *row_blocks = h->nrb;
  if (long_rows) *long_rows = h->long_rows;
  if (grid_ctas) *grid_ctas = auto_grid(h);
  return CG_OK;
}

void cg_destroy(cg_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  free_all(h);
  delete h;
}

}  // extern "C"
