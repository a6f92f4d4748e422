// The CG loop of small systems inside one thread-block cluster (CG_OPT_LOOP_MODE
// 4; automatic for small fp64 systems).  Alg. 1 with the stopping rule, true
// residual and restarts of cg_solve (readings R1-R5), on the caller's CSR.
//
// GB300 design.  A system of up to kClusterMax x kMaxRowsPerCta rows is split
// into equal row ranges, one per CTA of a cluster (up to 16 CTAs on 16 SMs of
// one GPC).  Each CTA keeps its rows of x, r, z = D^-1 r, two p buffers, q and
// D^-1 in shared memory; the SpMV reads other CTAs' entries through
// distributed shared memory (the owner of column j is floor(j / rows per CTA)).
// Dot products: each CTA stores its fixed-order block sum; after the hardware
// cluster barrier warp 0 of every CTA adds the partials of all CTAs in a fixed
// order and thread 0 forms the scalars and takes the loop decisions, so every
// CTA holds the same scalars and takes the same decisions (GB300's fp64 pipe
// issues 2 lanes a clock: scalar work done by all threads costs microseconds).  One
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
constexpr int kMinRowsPerCta = 64;   // small systems still spread over 16 SMs (fp64 issue per SM)
constexpr int kMaxRowsPerCta = 2048;  // 7 vectors x 2048 rows x 8 B = 112 KB of shared memory
constexpr int kCParts = 8;          // partial slots: 0 p.q, 1-2 (r.z, r.r), 4-6 residual (r.z, r.r, b.b)

struct ClusterParams {
  int n;
  int R;            // rows per CTA (the last CTA may hold fewer)
  unsigned rmagic;  // ceil(2^32 / R): the owner of column j is umulhi(j, rmagic)
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

// This CTA's block sums of v, pushed into every CTA's partial table (row =
// this CTA's rank, slots [slot, slot + NV)) by lanes 0..C-1 of warp 0 before
// the cluster barrier, so that after it each CTA reads the partials from its
// own shared memory (no remote load on the reduction's critical path).
// Block sums for the cluster form, where latency rules (about one row a
// thread): an xor tree in every warp at once, then warp 0 adds the 8 warp sums
// as a 3-level tree: 8 dependent fp64 adds instead of 12 (each costs ~80 clocks
// on GB300's fp64 pipe).  The result is in every lane of warp 0.
template <int NV>
__device__ __forceinline__ void cluster_block_sum(double (&v)[NV]) {
  __shared__ double s_w[NV][kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  }
  __syncthreads();  // warp 0 of the previous call has read s_w
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) s_w[j][warp] = v[j];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double a = lane < kWarps ? s_w[j][lane] : 0.0;
#pragma unroll
      for (int o = kWarps / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      v[j] = __shfl_sync(0xffffffffu, a, 0);
    }
  }
}

template <int NV>
__device__ __forceinline__ void put_partials(double (&v)[NV], double* const* rpart, int rank, int C, int slot) {
  cluster_block_sum<NV>(v);  // warp 0 holds the block sums in every lane
  if (threadIdx.x < C) {
    double* dst = rpart[threadIdx.x] + rank * kCParts + slot;
#pragma unroll
    for (int j = 0; j < NV; ++j) dst[j] = v[j];
  }
}

// After a cluster barrier, in warp 0: the partials of every CTA added in a fixed
// order.  Lane k takes CTA k's partial from this CTA's table, lanes C..31 hold
// 0, and a 4-level xor tree over lanes 0-15 forms the sum.  Every CTA holds the
// same partials, so every CTA gets the same bits.  Only warp 0 spends fp64
// issue slots on it (the pipe takes 2 lanes a clock).
template <int NV>
__device__ __forceinline__ void warp_cluster_sums(const double* part, int C, int slot, double (&out)[NV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double v = lane < C ? part[lane * kCParts + slot + j] : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    out[j] = v;
  }
}

// The CTA holding row j: floor(j / R) as a multiply-high.  With rmagic =
// floor(2^32 / R) + 1 the product overshoots j / R by less than j / 2^32 <
// 2^-17, while j / R lies at least 1 / R >= 2^-11 below the next integer, so the
// floor is exact for every row of a cluster system.
__device__ __forceinline__ int owner(const ClusterParams& P, int j) { return (int)__umulhi((unsigned)j, P.rmagic); }

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
  const int R = P.R;
  extern __shared__ __align__(16) double sm[];
  double* xs = sm;          // x of this CTA's rows
  double* rs = xs + R;      // r
  double* zs = rs + R;      // z = D^-1 r (r without Jacobi)
  double* pb0 = zs + R;     // two direction buffers
  double* pb1 = pb0 + R;
  double* qs = pb1 + R;     // A p
  double* dv = qs + R;      // 1 / A_ii
  double* part = dv + R;    // kClusterMax x kCParts partial sums, row = source CTA
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
  // The loop control (scalars, divisions, square roots, tests) runs in thread 0
  // of every CTA on the cluster-wide sums; the other threads follow the
  // broadcast words.  Thread 0 of every CTA takes the same decisions.
  __shared__ double s_alpha, s_beta;
  __shared__ int s_go;   // inner loop: 1 = run the next phase
  __shared__ int s_act;  // outer loop: 0 = leave, 1 = iterate, 2 = leave with x = 0
  __shared__ int s_act2; // after the inner loop: 0 = leave, 1 = recompute the true residual
  if (t == 0) s_beta = 0.0;
  int status = kNotConverged, k = 0, restarts = 0, k_before = 0, st_in = kNotConverged;
  double relres_true = 0.0, rr = 0.0, rr0 = 0.0, bb = 0.0, rho = 0.0, stop = 0.0, stop2_hi = 0.0;
  bool first = true, was_first = false, report_only = false;
  int par = 0;  // every thread: which buffer holds the current direction
  for (;;) {
    // residual r = b - A x (every CTA's x complete; the residual slots free), z, p = z
    cl.sync();
    double v3[3] = {0.0, 0.0, 0.0};
    for (int i = r0 + t; i < r1; i += kBlock) {
      const double s = row_dot(P, i, [&](int j) {
        const int o = owner(P, j);
        return s_x[o][j - o * R];
      });
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
    put_partials<3>(v3, s_part, rank, C, 4);
    cl.sync();
    if (t < 32) {
      double s3[3];
      warp_cluster_sums<3>(part, C, 4, s3);
      if (t == 0) {
        int act = 1;
        if (report_only) {  // breakdown / numeric error: the true residual of the last iterate
          relres_true = sqrt(s3[1]) / sqrt(bb);
          act = 0;
        } else if (first) {
          bb = s3[2];
          if (bb == 0.0) {  // b = 0: x = 0 solves it
            status = kOk;
            act = 2;
          }
        } else {
          relres_true = sqrt(s3[1]) / sqrt(bb);
          if (!isfinite(relres_true)) { status = kNumeric; act = 0; }
          else if (relres_true <= P.tol) { status = kOk; act = 0; }
          else if (k >= P.maxit || restarts >= P.max_restarts) { status = kNotConverged; act = 0; }
          else ++restarts;
        }
        int go = 0;
        if (act == 1) {
          was_first = first;
          first = false;
          rho = s3[0];
          rr = rr0 = s3[1];
          stop = P.tol * sqrt(bb);
          stop2_hi = stop2_high(stop);
          k_before = k;
          st_in = kNotConverged;
          if (below_stop(rr, stop, stop2_hi)) st_in = kOk;  // a4, before every SpMV
          else if (k < P.maxit) go = 1;
        }
        s_act = act;
        s_go = go;
      }
    }
    __syncthreads();
    const int act = s_act;
    if (act == 0) break;
    if (act == 2) {
      for (int i = r0 + t; i < r1; i += kBlock) xs[i - r0] = 0.0;
      break;
    }
    bool pending = false;  // p = z + beta p_old is due in the next phase A
    while (s_go) {
      // ---- A: p = z + beta p_old (own rows and, recomputed, the neighbours'), q = A p, p.q
      const double beta = s_beta;
      const double* po = par ? pb1 : pb0;
      double* pn = par ? pb0 : pb1;
      double* const* rpo = par ? s_p1 : s_p0;
      double v1[1] = {0.0};
      for (int i = r0 + t; i < r1; i += kBlock) {
        const int li = i - r0;
        const double pi = pending ? fma(beta, po[li], zs[li]) : po[li];
        const double q = pending ? row_dot(P, i,
                                           [&](int j) {
                                             const int o = owner(P, j), l = j - o * R;
                                             return fma(beta, rpo[o][l], s_z[o][l]);
                                           })
                                 : row_dot(P, i, [&](int j) {
                                     const int o = owner(P, j);
                                     return rpo[o][j - o * R];
                                   });
        if (pending) pn[li] = pi;
        qs[li] = q;
        v1[0] = fma(pi, q, v1[0]);
      }
      put_partials<1>(v1, s_part, rank, C, 0);
      cl.sync();
      if (t < 32) {
        double pq[1];
        warp_cluster_sums<1>(part, C, 0, pq);
        if (t == 0) {
          int go = 0;
          if (!isfinite(pq[0]) || !isfinite(rho)) st_in = kNumeric;
          else if (pq[0] <= 0.0) st_in = kBreakdown;
          else {
            s_alpha = rho / pq[0];
            go = 1;
          }
          s_go = go;
        }
      }
      __syncthreads();
      if (pending) par ^= 1;  // the new direction is current
      pending = false;
      if (!s_go) break;
      // ---- B: x += alpha p, r -= alpha q, z = D^-1 r; r.z, r.r
      const double alpha = s_alpha;
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
      put_partials<2>(v2, s_part, rank, C, 1);
      cl.sync();
      if (t < 32) {
        double s2[2];
        warp_cluster_sums<2>(part, C, 1, s2);
        if (t == 0) {
          s_beta = s2[0] / rho;
          rho = s2[0];
          rr = s2[1];
          ++k;
          int go = 0;
          if (below_stop(rr, stop, stop2_hi)) st_in = kOk;  // a4, before every SpMV
          else if (k < P.maxit) go = 1;
          s_go = go;
        }
      }
      __syncthreads();
      pending = true;
    }
    if (t == 0) {
      int act2 = 1;  // 1: loop back to recompute the true residual
      if (st_in == kNumeric || st_in == kBreakdown) {  // x keeps the last iterate; report its residual
        status = st_in;
        report_only = true;
      } else if (was_first && k == k_before && st_in == kOk) {  // x0 met tol: its true residual is known
        relres_true = sqrt(rr0) / sqrt(bb);
        status = kOk;
        act2 = 0;
      }
      s_act2 = act2;
    }
    __syncthreads();
    if (s_act2 == 0) break;
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

// CTAs and rows per CTA for n rows with clusters of at most cmax CTAs: as many
// CTAs as hold at least kMinRowsPerCta rows each (GB300 issues 2 fp64 lanes a
// clock per SM, so small systems go over as many SMs as the cluster has).
void cluster_shape(int64_t n, int cmax, int* rows, int* ctas) {
  const int64_t c = std::max<int64_t>(1, std::min<int64_t>(cmax, n / kMinRowsPerCta));
  *rows = (int)((n + c - 1) / c);
  *ctas = (int)((n + *rows - 1) / *rows);
}

size_t cluster_smem(int rows) { return sizeof(double) * ((size_t)7 * (size_t)rows + kClusterMax * kCParts); }

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
  int rows = 0, ctas = 0;
  for (;;) {
    cluster_shape(h->n, cmax, &rows, &ctas);
    if (rows > kMaxRowsPerCta) return (h->err = "cg_solve: system too large for the cluster form", CG_ERR_INVALID);
    const size_t smem = cluster_smem(rows);
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
    P.R = rows;
    P.rmagic = (unsigned)((1ull << 32) / (unsigned long long)rows + 1ull);
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
  for (int j = 0; j < 6; ++j) h->last.phase_ms[j] = ds.tphase[j] * 1e-6;
  h->last.kernel_launches = 1;
  const int64_t n = h->n, nnz = h->nnz;
  h->last.bytes_moved = (12 * nnz + 4 * (n + 1) + (jac ? 104 : 88) * n) * (int64_t)ds.iters;
  h->last.kernel_bytes_per_iter = 12 * nnz + 4 * (n + 1);  // the CSR from L1/L2; vectors stay on chip
  if (iters_out) *iters_out = ds.iters;
  if (relres_out) *relres_out = ds.relres_true;
  if (status < 0) h->err = std::string("cg_solve: ") + cg_status_string(status);
  return status;
}
