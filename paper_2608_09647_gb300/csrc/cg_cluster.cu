// The CG loop of small systems inside one thread-block cluster (CG_OPT_LOOP_MODE
// 4; automatic for small fp64 systems).  Alg. 1 with the stopping rule, true
// residual and restarts of cg_solve (readings R1-R5), on the caller's CSR.
//
// GB300 design.  A system of up to kClusterMax x kMaxRowsPerCta rows is split
// into power-of-two row ranges, one per CTA of a cluster (up to 16 CTAs on 16
// SMs of one GPC).  Each CTA keeps its rows of x, r, z = D^-1 r, two p buffers,
// q and D^-1 in shared memory; the SpMV reads other CTAs' entries through
// distributed shared memory (the owner of column j is j >> log2(rows per CTA)).
// Dot products: each CTA stores its fixed-order block sum, and after the
// hardware cluster barrier every CTA adds the partials of all CTAs in rank order,
// so every CTA holds the same scalars and takes the same decisions.  One
// iteration has two cluster barriers: phase A forms p = z + beta p_old for its
// rows (the neighbours' values recomputed from z and p_old, so p needs no
// barrier of its own) and q = A p with p.q; phase B updates x, r, z and forms
// r.z and r.r.  The system never leaves the SMs' shared memory between
// iterations; the matrix stays in L1/L2.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "cg_handle.cuh"

namespace cgx = cooperative_groups;
using namespace cg;

namespace {

constexpr int kClusterMax = 16;     // CTAs of the largest cluster (a non-portable size)
constexpr int kMinRowsPerCta = 256;
constexpr int kMaxRowsPerCta = 2048;  // 7 vectors x 2048 rows x 8 B = 112 KB of shared memory
constexpr int kCParts = 8;          // partial slots: 0 p.q, 1-2 (r.z, r.r), 4-6 residual (r.z, r.r, b.b)

struct ClusterParams {
  int n;
  int rshift;  // log2 of the rows per CTA
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ colind;
  const double* __restrict__ vals;
  const double* __restrict__ diag;  // A_ii (Jacobi)
  const double* __restrict__ b;
  double* x;
  double tol;
  int maxit, max_restarts, jac;
  DevState* st;
};

// This CTA's block sums of v into its partial slots [slot, slot + NV).
template <int NV>
__device__ __forceinline__ void put_partials(double (&v)[NV], double* part, int slot) {
  cta_sum0<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) part[slot + j] = v[j];
  }
}

// After a cluster barrier: the partials of every CTA added in rank order.  Lane
// k of each warp reads CTA k's partial (one remote load per lane, all in
// flight together); the lanes' values are then added in rank order through
// shuffles, so every thread of every CTA gets the same bits.
template <int NV>
__device__ __forceinline__ void cluster_sums(double* const* rpart, int C, int slot, double (&out)[NV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const double mine = lane < C ? rpart[lane][slot + j] : 0.0;
    double s = 0.0;
    for (int k = 0; k < C; ++k) s += __shfl_sync(0xffffffffu, mine, k);
    out[j] = s;
  }
}

constexpr int kGather = 8;  // a row's nonzeros whose remote loads are in flight together

// sum_k vals[k] v(colind[k]) over row i in storage order, with fused multiply-adds;
// v(j) reads the owner CTA's shared memory (every load of a chunk issued first)
template <class Vj>
__device__ __forceinline__ double row_dot(const ClusterParams& P, int i, Vj v) {
  const int a = __ldg(P.rowptr + i), e = __ldg(P.rowptr + i + 1);
  double s = 0.0;
  for (int k = a; k < e; k += kGather) {
    double av[kGather], xv[kGather];
#pragma unroll
    for (int u = 0; u < kGather; ++u) {
      const bool in = k + u < e;
      av[u] = in ? __ldg(P.vals + k + u) : 0.0;
      xv[u] = in ? v(__ldg(P.colind + k + u)) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kGather; ++u)
      if (k + u < e) s = fma(av[u], xv[u], s);
  }
  return s;
}

__global__ void __launch_bounds__(kBlock, 1) pcg_cluster_kernel(ClusterParams P) {
  cgx::cluster_group cl = cgx::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const int R = 1 << P.rshift;
  const int lmask = R - 1;
  extern __shared__ __align__(16) double sm[];
  double* xs = sm;          // x of this CTA's rows
  double* rs = xs + R;      // r
  double* zs = rs + R;      // z = D^-1 r (r without Jacobi)
  double* pb0 = zs + R;     // two direction buffers
  double* pb1 = pb0 + R;
  double* qs = pb1 + R;     // A p
  double* dv = qs + R;      // 1 / A_ii
  double* part = dv + R;    // kCParts partial sums
  __shared__ double* s_x[kClusterMax];  // every CTA's x, z, p buffers and partials
  __shared__ double* s_z[kClusterMax];
  __shared__ double* s_p0[kClusterMax];
  __shared__ double* s_p1[kClusterMax];
  __shared__ double* s_part[kClusterMax];
  const int t = threadIdx.x;
  if (t < C) {
    s_x[t] = cl.map_shared_rank(xs, t);
    s_z[t] = cl.map_shared_rank(zs, t);
    s_p0[t] = cl.map_shared_rank(pb0, t);
    s_p1[t] = cl.map_shared_rank(pb1, t);
    s_part[t] = cl.map_shared_rank(part, t);
  }
  const int n = P.n;
  const int r0 = rank * R;
  const int r1 = min(n, r0 + R);
  for (int i = r0 + t; i < r1; i += kBlock) {
    xs[i - r0] = P.x[i];
    dv[i - r0] = P.jac ? 1.0 / P.diag[i] : 1.0;
  }
  int status = kNotConverged, k = 0, restarts = 0, par = 0;
  double relres_true = 0.0, rr = 0.0, bb = 0.0;
  bool first = true, report_only = false;
  for (;;) {
    // residual r = b - A x (every CTA's x complete; the residual slots free), z, p = z
    cl.sync();
    double v3[3] = {0.0, 0.0, 0.0};
    for (int i = r0 + t; i < r1; i += kBlock) {
      const double s = row_dot(P, i, [&](int j) { return s_x[j >> P.rshift][j & lmask]; });
      const double bi = P.b[i];
      const double ri = bi - s;
      const double zi = dv[i - r0] * ri;
      rs[i - r0] = ri;
      zs[i - r0] = zi;
      pb0[i - r0] = zi;
      v3[0] = fma(ri, zi, v3[0]);
      v3[1] = fma(ri, ri, v3[1]);
      v3[2] = fma(bi, bi, v3[2]);
    }
    par = 0;
    put_partials<3>(v3, part, 4);
    cl.sync();
    double s3[3];
    cluster_sums<3>(s_part, C, 4, s3);
    if (report_only) {  // breakdown / numeric error: the true residual of the last iterate
      relres_true = sqrt(s3[1]) / sqrt(bb);
      break;
    }
    if (first) {
      bb = s3[2];
      if (bb == 0.0) {  // b = 0: x = 0 solves it
        for (int i = r0 + t; i < r1; i += kBlock) xs[i - r0] = 0.0;
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
    double rho = s3[0], beta = 0.0;
    rr = s3[1];
    const double stop = P.tol * sqrt(bb);
    const int k_before = k;
    int st = kNotConverged;
    bool pending = false;  // p = z + beta p_old is due in the next phase A
    for (;;) {
      if (sqrt(rr) <= stop) { st = kOk; break; }  // a4, before every SpMV
      if (k >= P.maxit) break;
      // ---- A: p = z + beta p_old (own rows and, recomputed, the neighbours'), q = A p, p.q
      const double* po = par ? pb1 : pb0;
      double* pn = par ? pb0 : pb1;
      double* const* rpo = par ? s_p1 : s_p0;
      double v1[1] = {0.0};
      for (int i = r0 + t; i < r1; i += kBlock) {
        const int li = i - r0;
        const double pi = pending ? fma(beta, po[li], zs[li]) : po[li];
        const double q = pending ? row_dot(P, i,
                                           [&](int j) {
                                             const int o = j >> P.rshift, l = j & lmask;
                                             return fma(beta, rpo[o][l], s_z[o][l]);
                                           })
                                 : row_dot(P, i, [&](int j) { return rpo[j >> P.rshift][j & lmask]; });
        if (pending) pn[li] = pi;
        qs[li] = q;
        v1[0] = fma(pi, q, v1[0]);
      }
      put_partials<1>(v1, part, 0);
      cl.sync();
      double pq[1];
      cluster_sums<1>(s_part, C, 0, pq);
      if (pending) par ^= 1;  // the new direction is current
      pending = false;
      if (!isfinite(pq[0]) || !isfinite(rho)) { st = kNumeric; break; }
      if (pq[0] <= 0.0) { st = kBreakdown; break; }
      const double alpha = rho / pq[0];
      // ---- B: x += alpha p, r -= alpha q, z = D^-1 r; r.z, r.r
      const double* pc = par ? pb1 : pb0;
      double v2[2] = {0.0, 0.0};
      for (int i = r0 + t; i < r1; i += kBlock) {
        const int li = i - r0;
        xs[li] = fma(alpha, pc[li], xs[li]);
        const double ri = fma(-alpha, qs[li], rs[li]);
        const double zi = dv[li] * ri;
        rs[li] = ri;
        zs[li] = zi;
        v2[0] = fma(ri, zi, v2[0]);
        v2[1] = fma(ri, ri, v2[1]);
      }
      put_partials<2>(v2, part, 1);
      cl.sync();
      double s2[2];
      cluster_sums<2>(s_part, C, 1, s2);
      beta = s2[0] / rho;
      rho = s2[0];
      rr = s2[1];
      ++k;
      pending = true;
    }
    if (st == kNumeric || st == kBreakdown) {  // x keeps the last iterate; report its residual
      status = st;
      report_only = true;
      continue;
    }
    if (was_first && k == k_before && st == kOk) {  // x0 met tol: its true residual is s3[1]
      relres_true = sqrt(s3[1]) / sqrt(bb);
      status = kOk;
      break;
    }
    // kOk or kNotConverged: loop back to recompute the true residual
  }
  for (int i = r0 + t; i < r1; i += kBlock) P.x[i] = xs[i - r0];
  if (rank == 0 && t == 0) {
    P.st->status = status;
    P.st->iters = k;
    P.st->restarts = restarts;
    P.st->relres_true = relres_true;
    P.st->relres_rec = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Rows per CTA (a power of two) and CTAs for n rows with clusters of at most cmax CTAs.
void cluster_shape(int64_t n, int cmax, int* rshift, int* ctas) {
  int s = 0;
  while ((1 << s) < kMinRowsPerCta) ++s;
  while ((int64_t)(1 << s) * cmax < n) ++s;
  *rshift = s;
  *ctas = (int)std::max<int64_t>(1, (n + (1 << s) - 1) >> s);
}

size_t cluster_smem(int rshift) { return sizeof(double) * ((size_t)7 * ((size_t)1 << rshift) + kCParts); }

}  // namespace

int64_t cgi::cluster_max_rows() { return (int64_t)kClusterMax * kMaxRowsPerCta; }

cg_status cgi::cluster_solve(cg_handle* h, const double* b, double* x, double tol, int32_t maxit, bool jac,
                             int32_t* iters_out, double* relres_out) {
  if (h->n > cluster_max_rows()) {
    h->err = "cg_solve: the cluster loop form holds at most " + std::to_string(cluster_max_rows()) + " rows";
    return CG_ERR_INVALID;
  }
  auto cuda_err = [&](cudaError_t e, const char* where) {
    h->err = std::string("cg_solve (cluster form): ") + where + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CG_ERR_OOM : CG_ERR_CUDA;
  };
  // the largest cluster the device can place: 16 CTAs (non-portable), else 8
  int cmax = kClusterMax;
  cudaError_t e = cudaFuncSetAttribute(pcg_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cmax = 8;
  }
  int rshift = 0, ctas = 0;
  for (;;) {
    cluster_shape(h->n, cmax, &rshift, &ctas);
    if (rshift > 11) return (h->err = "cg_solve: system too large for the cluster form", CG_ERR_INVALID);
    const size_t smem = cluster_smem(rshift);
    e = cudaFuncSetAttribute(pcg_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_err(e, "shared memory size");
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int active = 0;
    e = cudaOccupancyMaxActiveClusters(&active, pcg_cluster_kernel, &cfg);
    if ((e != cudaSuccess || active < 1) && cmax > 8) {  // fall back to the portable size
      cudaGetLastError();
      cmax = 8;
      continue;
    }
    if (e != cudaSuccess) return cuda_err(e, "cluster occupancy");
    if (active < 1) return (h->err = "cg_solve: no cluster of this size fits the device", CG_ERR_CUDA);
    ClusterParams P{};
    P.n = (int)h->n;
    P.rshift = rshift;
    P.rowptr = h->rowptr;
    P.colind = h->colind;
    P.vals = h->vals;
    P.diag = h->diag;
    P.b = b;
    P.x = x;
    P.tol = tol;
    P.maxit = maxit;
    P.max_restarts = h->max_restarts;
    P.jac = jac ? 1 : 0;
    P.st = h->st;
    if ((e = cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream)) != cudaSuccess) return cuda_err(e, "memset");
    if ((e = cudaEventRecord(h->ev0, h->stream)) != cudaSuccess) return cuda_err(e, "event");
    if ((e = cudaLaunchKernelEx(&cfg, pcg_cluster_kernel, P)) != cudaSuccess) return cuda_err(e, "launch");
    if ((e = cudaEventRecord(h->ev1, h->stream)) != cudaSuccess) return cuda_err(e, "event");
    if ((e = cudaMemcpyAsync(h->host_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
      return cuda_err(e, "status copy");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_err(e, "synchronize");
    break;
  }
  float ms = 0.0f;
  if ((e = cudaEventElapsedTime(&ms, h->ev0, h->ev1)) != cudaSuccess) return cuda_err(e, "event time");
  const DevState& ds = *h->host_st;
  const cg_status status = (cg_status)ds.status;
  h->last.status = status;
  h->last.iters = ds.iters;
  h->last.restarts = ds.restarts;
  h->last.grid_ctas = ctas;
  h->last.relres_true = ds.relres_true;
  h->last.relres_rec = ds.relres_rec;
  h->last.kernel_ms = ms;
  h->last.loop_form = 4;
  h->last.kernel_launches = 1;
  const int64_t n = h->n, nnz = h->nnz;
  h->last.bytes_moved = (12 * nnz + 4 * (n + 1) + (jac ? 104 : 88) * n) * (int64_t)ds.iters;
  h->last.kernel_bytes_per_iter = 12 * nnz + 4 * (n + 1);  // the CSR from L1/L2; vectors stay on chip
  if (iters_out) *iters_out = ds.iters;
  if (relres_out) *relres_out = ds.relres_true;
  if (status < 0) h->err = std::string("cg_solve: ") + cg_status_string(status);
  return status;
}
