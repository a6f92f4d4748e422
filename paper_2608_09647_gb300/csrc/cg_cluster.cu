// The CG loop of small systems inside one thread-block cluster (CG_OPT_LOOP_MODE
// 4; automatic for small fp64 systems).  Alg. 1 with the stopping rule, true
// residual and restarts of cg_solve (readings R1-R5), on the caller's CSR.
//
// GB300 design.  A system of up to kClusterMax x kMaxRowsPerCta rows is split
// into equal row ranges, one per CTA of a cluster (up to 16 CTAs on 16 SMs of
// one GPC).  Each CTA keeps its rows of x, r, z = D^-1 r, two p buffers, q and
// D^-1 in shared memory and, when it fits, its rows of the CSR too, with every
// column turned into the distributed-shared-memory address of that entry of x
// in its owner CTA (the owner of column j is floor(j / rows per CTA)).  The
// loop never touches global memory: a global load costs ~170 clocks even when
// it hits L1, and every cluster-scope acquire sends the next one to L2.
//
// Dot products: each CTA sums its threads' values exactly on the integer pipes
// (cg_exact.cuh: each warp at its own scale, then warp 0 over the 8 warp sums)
// and pushes the sum into a slot table of every CTA with st.async, whose bytes
// complete a transaction count on the receiving CTA's mbarrier; each CTA waits
// (bounded) on its own mbarrier, then warp 0 adds the C entries exactly and
// rounds once, and thread 0 forms the scalars and takes the loop decisions, so
// every CTA holds the same scalars and takes the same decisions.  An exchange
// costs ~830 clocks where remote stores and a cluster barrier took ~1,270; the
// two slot tables and mbarriers alternate, so a CTA can run one exchange ahead.
//
// One iteration has two exchanges.  Phase A forms p = z + beta p_old for its
// rows, then q = A p and p.q; a neighbour in another CTA has its p recomputed
// from that CTA's z and p_old (the same bits), so p needs no exchange of its
// own.  Phase B updates r and z and forms r.z and r.r; x += alpha p runs after
// the push, while the partials are in flight.  The true residual reads other
// CTAs' x, so it follows an exchange with no payload that every CTA makes after
// its last x update.  GB300's fp64 unit issues one warp instruction per ~64
// clocks per SM sub-partition, so fp64 work is kept to what the iteration
// needs: no fp64 in the sums, scalars in thread 0 (1 / rho in warp 1, off the
// path), and the recomputed p only in warps that hold a neighbour of another CTA.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "cg_exact.cuh"
#include "cg_handle.cuh"

namespace cgx = cooperative_groups;
using namespace cg;

namespace {

constexpr int kClusterMax = 16;      // CTAs of the largest cluster (a non-portable size)
constexpr int kMinRowsPerCta = 64;   // small systems still spread over 16 SMs (fp64 issue per SM)
constexpr int kMaxRowsPerCta = 2048; // 7 vectors x 2048 rows x 8 B = 112 KB of shared memory
constexpr int kSlots = 3;            // values a warp pushes per exchange
constexpr int kGather = 8;           // a row's entries whose loads are in flight together
constexpr int kVec = 7;              // vectors per CTA: x, r, z, p0, p1, q, D^-1

struct ClusterParams {
  int n;
  int R;            // rows per CTA (the last CTA may hold fewer)
  unsigned rmagic;  // floor(2^32 / R) + 1: the owner of column j is umulhi(j, rmagic)
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ colind;
  const double* __restrict__ vals;
  const double* __restrict__ diag;  // A_ii (Jacobi)
  const double* __restrict__ b;
  double* x;
  double tol;
  int maxit, max_restarts, jac;
  uint64_t timeout_ns;  // limit of every wait for an exchange
  unsigned skip_seq;    // fault injection: CTA 0 does not push exchange #skip_seq (1-based)
  DevState* st;
};

// ---- distributed shared memory and mbarrier primitives (PTX ISA 8.x, sm_90+)

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// the address of this CTA's shared-memory location `a` in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cluster_addr(unsigned a, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

// The "memory" clobber keeps the load after the barrier or exchange wait that
// makes its data current: with the address in a register nothing else orders it.
__device__ __forceinline__ double ld_dsmem(unsigned a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// this thread's arrival, announcing `bytes` of st.async payload for the current phase
__device__ __forceinline__ void mbar_arrive_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// st.async of 16 bytes into another CTA's shared memory, completing them on that
// CTA's mbarrier (`dst` and `rbar` are cluster addresses)
__device__ __forceinline__ void st_async_v2u64(unsigned dst, unsigned long long v0, unsigned long long v1,
                                               unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.u64 [%0], {%1, %2}, [%3];" ::"r"(dst),
               "l"(v0), "l"(v1), "r"(rbar)
               : "memory");
}

// ---- exchanges

// Shared state of the exchanges (static shared memory: the same offsets in every
// CTA).  An entry holds an exact integer sum with its scale (cg_exact::pack).
struct Exchange {
  ulonglong2 part[2][kClusterMax][kSlots];  // [parity][source CTA][value]: the CTAs' sums
  ulonglong2 warp[kWarps][kSlots];          // this CTA's warp sums
  unsigned long long bar[2];                // mbarrier per parity: 1 arrival + the pushed bytes
};

// This CTA's NV sums, exact and order-free, pushed by lanes 0..C-1 of warp 0 into
// row `rank` of slot table `par` of CTA `lane`.  Every warp first sums its lanes'
// values at the warp's own scale (the largest exponent among them); warp 0 then
// adds the 8 warp sums at the CTA's scale.  No fp64 instruction is involved.
template <int NV>
__device__ __forceinline__ void push_sums(const double (&v)[NV], Exchange& X, int rank, int C, int par, bool skip) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const ulonglong2 w = warp_exact(v[j]);
    if (lane == 0) X.warp[warp][j] = w;
  }
  __syncthreads();  // every warp's sums, and the CTA's stores of this phase, before the push
  if (warp == 0) {
    unsigned long long lo[NV], hi[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      int E;
      bool bad;
      const cg_exact::i128 S = sum_entries(X.warp[lane < kWarps ? lane : 0][j], lane < kWarps, &E, &bad);
      cg_exact::pack(S, E, bad, &lo[j], &hi[j]);
    }
    if (lane < C && !skip) {
      const unsigned rbar = cluster_addr(smem_addr(&X.bar[par]), (unsigned)lane);
#pragma unroll
      for (int j = 0; j < NV; ++j)
        st_async_v2u64(cluster_addr(smem_addr(&X.part[par][rank][j]), (unsigned)lane), lo[j], hi[j], rbar);
    }
  }
}

// Called by every lane of warp 0: wait until every CTA has pushed exchange `e`
// (0-based) into this CTA's table.  Exchange e uses table and
// mbarrier e & 1; it is that mbarrier's (e >> 1)-th phase.  The wait gives up
// after timeout_ns (false in every lane).
__device__ __forceinline__ bool wait_sums(Exchange& X, unsigned e, uint64_t timeout_ns) {
  const unsigned bar = smem_addr(&X.bar[e & 1u]), parity = (e >> 1) & 1u;
  bool ok = false;
  uint64_t t0 = 0;
  for (unsigned spins = 0;; ++spins) {
    if (mbar_try_wait(bar, parity)) {
      ok = true;
      break;
    }
    if (spins == 0) t0 = global_timer_ns();
    else if ((spins & 15u) == 0u && global_timer_ns() - t0 > timeout_ns) break;
  }
  return __all_sync(0xffffffffu, ok);
}

// In warp 0 after wait_sums: the C CTA sums of each value (lane k takes CTA k's)
// moved to their largest scale, added exactly and rounded once to fp64.  Every
// CTA holds the same entries, so every CTA gets the same bits.
template <int NV>
__device__ __forceinline__ void cluster_sums(const Exchange& X, int par, int C, double (&out)[NV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    int E;
    bool bad;
    const cg_exact::i128 T = sum_entries(X.part[par][lane < C ? lane : 0][j], lane < C, &E, &bad);
    out[j] = cg_exact::to_fp64(T, E, bad);
  }
}

// ---- this CTA's rows of the CSR

// The CTA holding row j: floor(j / R) as a multiply-high.  With rmagic =
// floor(2^32 / R) + 1 the product overshoots j / R by less than j / 2^32 <
// 2^-17, while j / R lies at least 1 / R >= 2^-11 below the next integer, so the
// floor is exact for every row of a cluster system.
__device__ __forceinline__ int owner(const ClusterParams& P, int j) { return (int)__umulhi((unsigned)j, P.rmagic); }

// Rows held in shared memory: local row pointers, values and, per entry, the
// cluster address of the column's x entry in its owner CTA.
struct SliceSmem {
  const int* rp;
  const double* val;
  const unsigned* adr;
  __device__ __forceinline__ int start(int li) const { return rp[li]; }
  __device__ __forceinline__ int len(int li) const { return rp[li + 1] - rp[li]; }
  __device__ __forceinline__ double value(int k) const { return val[k]; }
  __device__ __forceinline__ unsigned address(int k) const { return adr[k]; }
};

// Rows too large for shared memory: the caller's CSR, the address formed per entry.
struct SliceGlobal {
  const int32_t* rp;      // the caller's row pointers from this CTA's first row
  const int32_t* col;
  const double* val;
  const unsigned* cbase;  // cluster address of x[0] in every CTA
  unsigned rmagic;
  int R;
  __device__ __forceinline__ int start(int li) const { return __ldg(rp + li); }
  __device__ __forceinline__ int len(int li) const { return __ldg(rp + li + 1) - __ldg(rp + li); }
  __device__ __forceinline__ double value(int k) const { return __ldg(val + k); }
  __device__ __forceinline__ unsigned address(int k) const {
    const int j = __ldg(col + k), o = (int)__umulhi((unsigned)j, rmagic);
    return cbase[o] + 8u * (unsigned)(j - o * R);
  }
};

// The vector a row product reads, as byte offsets from x's cluster address.
struct Operand {
  unsigned off;     // the vector read (x, or the current direction)
  unsigned off_po;  // pending update: p_old and z of other CTAs' rows
  unsigned off_z;
  unsigned own;     // cluster address of this CTA's x[0]
  unsigned span;    // 8 R: the entry is this CTA's when (address - own) < span
  double beta;
  bool pending;     // p = z + beta p_old not yet formed for other CTAs' rows
};

// The first row of a thread, its entries held in registers across iterations
// (the loop's smem loads of addresses and values leave the critical path).
struct RowRegs {
  unsigned a[kGather];
  double v[kGather];
  __device__ __forceinline__ unsigned address(int k) const { return a[k]; }
  __device__ __forceinline__ double value(int k) const { return v[k]; }
};

// One chunk (entries kc .. kc + kGather - 1) of sum_k val_k v(col_k) over a
// lane's row (len entries from k0), fused multiply-adds in storage order onto s.
// Every lane of the warp runs to the warp's longest row (nmax) with its sum held
// past its own end, so the warp votes stay converged.  With a pending direction,
// another CTA's entry is recomputed as fma(beta, p_old, z), only in warps that
// hold one.
template <class Slice>
__device__ __forceinline__ double row_chunk(const Slice& A, int k0, int len, int kc, int nmax, const Operand& O,
                                           double s) {
  double av[kGather], xv[kGather], zv[kGather];
  bool rem[kGather];
#pragma unroll
  for (int u = 0; u < kGather; ++u) {
    if (kc + u < nmax) {
      const bool in = kc + u < len;
      unsigned a = O.own;  // lanes past their row's end read this CTA's x[0], a valid address
      av[u] = 0.0;
      if (in) {
        a = A.address(k0 + kc + u);
        av[u] = A.value(k0 + kc + u);
      }
      rem[u] = O.pending && in && (a - O.own) >= O.span;
      xv[u] = ld_dsmem(a + (rem[u] ? O.off_po : O.off));
      zv[u] = rem[u] ? ld_dsmem(a + O.off_z) : 0.0;
    }
  }
#pragma unroll
  for (int u = 0; u < kGather; ++u) {
    if (kc + u < nmax) {
      if (O.pending && __any_sync(0xffffffffu, rem[u])) xv[u] = rem[u] ? fma(O.beta, xv[u], zv[u]) : xv[u];
      if (kc + u < len) s = fma(av[u], xv[u], s);
    }
  }
  return s;
}

template <class Slice>
__device__ __forceinline__ double row_dot(const Slice& A, int k0, int len, int nmax, const Operand& O) {
  double s = 0.0;
  for (int k = 0; k < nmax; k += kGather) s = row_chunk(A, k0, len, k, nmax, O, s);
  return s;
}

template <bool SMEM>
__global__ void __launch_bounds__(kBlock, 1) pcg_cluster_kernel(ClusterParams P) {
  cgx::cluster_group cl = cgx::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const int R = P.R;
  extern __shared__ __align__(16) double sm[];
  double* xs = sm;          // x of this CTA's rows
  double* rs = xs + R;      // r
  double* zb = rs + R;      // z = D^-1 r
  double* zs = P.jac ? zb : rs;  // plain CG: z is r (the z buffer stays unused)
  double* pb0 = zb + R;     // two direction buffers
  double* pb1 = pb0 + R;
  double* qs = pb1 + R;     // A p
  double* dv = qs + R;      // 1 / A_ii
  __shared__ Exchange X;
  __shared__ unsigned s_cb[kClusterMax];  // cluster address of x[0] in every CTA
  const int t = threadIdx.x;
  const int n = P.n;
  const int r0 = rank * R;
  const int nr = min(n, r0 + R) - r0;  // this CTA's rows
  const int nsl = (nr + kBlock - 1) / kBlock;
  if (t < C) s_cb[t] = cluster_addr(smem_addr(xs), (unsigned)t);
  for (int li = t; li < nr; li += kBlock) {
    xs[li] = P.x[r0 + li];
    dv[li] = P.jac ? 1.0 / P.diag[r0 + li] : 1.0;
  }
  if (t == 0) {
    mbar_init(smem_addr(&X.bar[0]), 1);
    mbar_init(smem_addr(&X.bar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  SliceSmem AS{};
  if (SMEM) {  // this CTA's rows of the CSR into shared memory, columns as cluster addresses
    int* lrp = reinterpret_cast<int*>(dv + R);
    double* lval = reinterpret_cast<double*>(lrp + ((R + 2) & ~1));
    const int k0 = P.rowptr[r0], k1 = P.rowptr[r0 + nr];
    unsigned* ladr = reinterpret_cast<unsigned*>(lval + (k1 - k0));
    for (int li = t; li <= nr; li += kBlock) lrp[li] = P.rowptr[r0 + li] - k0;
    for (int k = k0 + t; k < k1; k += kBlock) {
      const int j = P.colind[k], o = owner(P, j);
      lval[k - k0] = P.vals[k];
      ladr[k - k0] = s_cb[o] + 8u * (unsigned)(j - o * R);
    }
    AS = SliceSmem{lrp, lval, ladr};
  }
  const SliceGlobal AG{P.rowptr + r0, P.colind, P.vals, s_cb, P.rmagic, R};
  const unsigned own = s_cb[rank], span = 8u * (unsigned)R;
  const unsigned off_z = P.jac ? 2u * span : span, off_p0 = 3u * span;  // z; p buffer b at off_p0 + b span

  // every CTA's mbarriers initialised, every CTA's x and this CTA's CSR slice in
  // shared memory before any push, remote read or read of the slice
  cl.sync();
  // the first row of each thread in registers when the warp's rows have at most kGather entries
  RowRegs RC;
  int len0 = 0, nmax0 = 0;
  bool cached = false;
  if (SMEM) {
    int k0 = 0;
    if (t < nr) {
      len0 = AS.len(t);
      k0 = AS.start(t);
    }
    nmax0 = __reduce_max_sync(0xffffffffu, len0);
    cached = nmax0 <= kGather;
#pragma unroll
    for (int u = 0; u < kGather; ++u) {
      RC.a[u] = own;
      RC.v[u] = 0.0;
      if (u < len0) {
        RC.a[u] = AS.address(k0 + u);
        RC.v[u] = AS.value(k0 + u);
      }
    }
  }

  // The loop control (scalars, divisions, square roots, tests) runs in thread 0
  // of every CTA on the cluster-wide sums; the other threads follow the
  // broadcast words.  Thread 0 of every CTA takes the same decisions.
  __shared__ double s_alpha, s_beta;
  __shared__ double s_rho, s_inv_rho;  // rho (thread 0's), and 1 / rho formed by warp 1
  __shared__ int s_go;   // inner loop: 1 = run the next phase
  __shared__ int s_act;  // outer loop: 0 = leave, 1 = iterate, 2 = leave with x = 0
  __shared__ int s_act2; // after the inner loop: 0 = leave, 1 = recompute the true residual
  if (t == 0) s_beta = 0.0;
  int status = kNotConverged, k = 0, restarts = 0, k_before = 0, st_in = kNotConverged;
  double relres_true = 0.0, rr = 0.0, rr0 = 0.0, bb = 0.0, rho = 0.0, stop = 0.0, stop2_hi = 0.0;
  bool first = true, was_first = false, report_only = false;
  int par = 0;      // every thread: which buffer holds the current direction
  unsigned e = 0;   // every thread: exchanges made so far
  bool pass0 = true;
  const uint64_t tmo = P.timeout_ns;
  // every exchange: thread 0 arms this CTA's mbarrier, the CTA's exact sum is pushed,
  // warp 0 waits; on a timeout thread 0 records it and the CTA leaves
  auto arm = [&](int nv) {
    if (t == 0) mbar_arrive_expect(smem_addr(&X.bar[e & 1u]), (unsigned)(C * nv * 16));
  };
  auto record_timeout = [&]() {
    if (atomicCAS(&P.st->abort, 0, 1) == 0) {
      P.st->err_cta = (int)blockIdx.x;
      P.st->err_barrier = (int)e + 1;
    }
  };
  for (;;) {
    // the true residual reads every CTA's x: after the first pass, an exchange
    // with no payload that every CTA makes after its last x update
    if (!pass0) {
      arm(1);
      double v0[1] = {0.0};
      push_sums<1>(v0, X, rank, C, (int)(e & 1u), P.skip_seq == e + 1u && rank == 0);
      if (t < 32) {
        const bool ok = wait_sums(X, e, tmo);
        if (t == 0) {
          s_act = ok ? 1 : 0;
          if (!ok) { record_timeout(); status = kTimeout; }
        }
      }
      ++e;
      __syncthreads();
      if (s_act == 0) break;
    }
    pass0 = false;
    // residual r = b - A x, z, p = z
    arm(3);
    double v3[3] = {0.0, 0.0, 0.0};
    const Operand Ox{0u, 0u, 0u, own, span, 0.0, false};
    for (int sl = 0; sl < nsl; ++sl) {
      const int li = t + sl * kBlock;
      const bool valid = li < nr;
      double s;
      if (SMEM && sl == 0 && cached) {
        s = row_chunk(RC, 0, len0, 0, nmax0, Ox, 0.0);
      } else {
        int len = 0, k0 = 0;
        if (valid) {  // rows past this CTA's last one read nothing
          len = SMEM ? AS.len(li) : AG.len(li);
          k0 = SMEM ? AS.start(li) : AG.start(li);
        }
        const int nmax = __reduce_max_sync(0xffffffffu, len);
        s = SMEM ? row_dot(AS, k0, len, nmax, Ox) : row_dot(AG, k0, len, nmax, Ox);
      }
      if (valid) {
        const double bi = P.b[r0 + li];
        const double ri = bi - s;
        const double zi = P.jac ? dv[li] * ri : ri;
        rs[li] = ri;
        zs[li] = zi;
        pb0[li] = zi;
        v3[0] = fma(ri, zi, v3[0]);
        v3[1] = fma(ri, ri, v3[1]);
        v3[2] = fma(bi, bi, v3[2]);
      }
    }
    par = 0;
    push_sums<3>(v3, X, rank, C, (int)(e & 1u), P.skip_seq == e + 1u && rank == 0);
    if (t < 32) {
      const bool ok = wait_sums(X, e, tmo);
      double s3[3];
      cluster_sums<3>(X, (int)(e & 1u), C, s3);
      if (t == 0) {
        int act = 1;
        if (!ok) {
          record_timeout();
          status = kTimeout;
          act = 0;
        } else if (report_only) {  // breakdown / numeric error: the true residual of the last iterate
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
          s_rho = rho;
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
    ++e;
    __syncthreads();
    const int act = s_act;
    if (act == 0) break;
    if (act == 2) {
      for (int li = t; li < nr; li += kBlock) xs[li] = 0.0;
      break;
    }
    bool pending = false;  // p = z + beta p_old is due in the next phase A
    while (s_go) {
      // ---- A: p = z + beta p_old for this CTA's rows, q = A p (other CTAs' p
      // recomputed), p.q
      arm(1);
      const double beta = s_beta;
      const double* po = par ? pb1 : pb0;
      double* pn = par ? pb0 : pb1;
      if (pending) {
        for (int li = t; li < nr; li += kBlock) pn[li] = fma(beta, po[li], zs[li]);
        __syncthreads();  // this CTA's p complete before its rows' neighbours read it
      }
      const double* pc = pending ? pn : po;
      const unsigned off_po = off_p0 + (unsigned)par * span, off_pn = off_p0 + (unsigned)(par ^ 1) * span;
      const Operand Op{pending ? off_pn : off_po, off_po, off_z, own, span, beta, pending};
      double v1[1] = {0.0};
      for (int sl = 0; sl < nsl; ++sl) {
        const int li = t + sl * kBlock;
        const bool valid = li < nr;
        double q;
        if (SMEM && sl == 0 && cached) {
          q = row_chunk(RC, 0, len0, 0, nmax0, Op, 0.0);
        } else {
          int len = 0, k0 = 0;
          if (valid) {  // rows past this CTA's last one read nothing
            len = SMEM ? AS.len(li) : AG.len(li);
            k0 = SMEM ? AS.start(li) : AG.start(li);
          }
          const int nmax = __reduce_max_sync(0xffffffffu, len);
          q = SMEM ? row_dot(AS, k0, len, nmax, Op) : row_dot(AG, k0, len, nmax, Op);
        }
        if (valid) {
          qs[li] = q;
          v1[0] = fma(pc[li], q, v1[0]);
        }
      }
      push_sums<1>(v1, X, rank, C, (int)(e & 1u), P.skip_seq == e + 1u && rank == 0);
      // 1 / rho for this iteration's beta, on another SM sub-partition while warp 0
      // waits for p.q and forms alpha: beta = rho' (1 / rho) costs a multiply on
      // the path where rho' / rho cost a division (within 1.5 ulp of it)
      if (t == 32) s_inv_rho = 1.0 / s_rho;
      if (t < 32) {
        const bool ok = wait_sums(X, e, tmo);
        double pq[1];
        cluster_sums<1>(X, (int)(e & 1u), C, pq);
        if (t == 0) {
          int go = 0;
          if (!ok) {
            record_timeout();
            st_in = kTimeout;
          } else if (!isfinite(pq[0]) || !isfinite(rho)) st_in = kNumeric;
          else if (pq[0] <= 0.0) st_in = kBreakdown;
          else {
            s_alpha = rho / pq[0];
            go = 1;
          }
          s_go = go;
        }
      }
      ++e;
      __syncthreads();
      if (pending) par ^= 1;  // the new direction is current
      pending = false;
      if (!s_go) break;
      // ---- B: r -= alpha q, z = D^-1 r; r.z, r.r; then x += alpha p while they are in
      // flight (plain CG: z is r and r.z is r.r, one sum)
      arm(P.jac ? 2 : 1);
      const double alpha = s_alpha;
      const double* pcur = par ? pb1 : pb0;
      if (P.jac) {
        double v2[2] = {0.0, 0.0};
        for (int li = t; li < nr; li += kBlock) {
          const double ri = fma(-alpha, qs[li], rs[li]);
          const double zi = dv[li] * ri;
          rs[li] = ri;
          zs[li] = zi;
          v2[0] = fma(ri, zi, v2[0]);
          v2[1] = fma(ri, ri, v2[1]);
        }
        push_sums<2>(v2, X, rank, C, (int)(e & 1u), P.skip_seq == e + 1u && rank == 0);
      } else {
        double v2[1] = {0.0};
        for (int li = t; li < nr; li += kBlock) {
          const double ri = fma(-alpha, qs[li], rs[li]);
          rs[li] = ri;
          v2[0] = fma(ri, ri, v2[0]);
        }
        push_sums<1>(v2, X, rank, C, (int)(e & 1u), P.skip_seq == e + 1u && rank == 0);
      }
      for (int li = t; li < nr; li += kBlock) xs[li] = fma(alpha, pcur[li], xs[li]);
      if (t < 32) {
        const bool ok = wait_sums(X, e, tmo);
        double s2[2];
        if (P.jac) {
          cluster_sums<2>(X, (int)(e & 1u), C, s2);
        } else {
          double s1[1];
          cluster_sums<1>(X, (int)(e & 1u), C, s1);
          s2[0] = s2[1] = s1[0];
        }
        if (t == 0) {
          int go = 0;
          if (!ok) {
            record_timeout();
            st_in = kTimeout;
          } else {
            s_beta = s2[0] * s_inv_rho;
            rho = s2[0];
            s_rho = rho;
            rr = s2[1];
            ++k;
            if (below_stop(rr, stop, stop2_hi)) st_in = kOk;  // a4, before every SpMV
            else if (k < P.maxit) go = 1;
          }
          s_go = go;
        }
      }
      ++e;
      __syncthreads();
      pending = true;
    }
    if (t == 0) {
      int act2 = 1;  // 1: loop back to recompute the true residual
      if (st_in == kTimeout) {
        status = kTimeout;
        act2 = 0;
      } else if (st_in == kNumeric || st_in == kBreakdown) {  // x keeps the last iterate; report its residual
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
  for (int li = t; li < nr; li += kBlock) P.x[r0 + li] = xs[li];
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

// Dynamic shared memory of a CTA: the vectors, and with the CSR held in shared
// memory its row pointers (an even count) and, per entry, a value and an address.
size_t cluster_smem(int rows, int64_t slice_nnz) {
  size_t b = sizeof(double) * (size_t)kVec * (size_t)rows;
  if (slice_nnz >= 0) b += sizeof(int) * (size_t)((rows + 2) & ~1) + 12 * (size_t)slice_nnz;
  return b;
}

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
  int dev = 0, smem_optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return cuda_err(e, "device attributes");
  // the largest cluster the device can place: 16 CTAs (non-portable), else 8
  int cmax = kClusterMax;
  for (const void* fn : {(const void*)pcg_cluster_kernel<true>, (const void*)pcg_cluster_kernel<false>}) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      cmax = 8;
    }
  }
  int rows = 0, ctas = 0;
  bool csr_in_smem = false;
  for (;;) {
    cluster_shape(h->n, cmax, &rows, &ctas);
    if (rows > kMaxRowsPerCta) return (h->err = "cg_solve: system too large for the cluster form", CG_ERR_INVALID);
    // the CSR goes to shared memory when the largest CTA slice fits beside the vectors
    int64_t slice = 0;
    const std::vector<int32_t>& rp = h->host_rowptr;
    for (int c = 0; c < ctas; ++c) {
      const int64_t a = (int64_t)c * rows, z = std::min<int64_t>(h->n, a + rows);
      slice = std::max<int64_t>(slice, (int64_t)rp[(size_t)z] - rp[(size_t)a]);
    }
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, (const void*)pcg_cluster_kernel<true>)) != cudaSuccess)
      return cuda_err(e, "kernel attributes");
    const bool in_smem = cluster_smem(rows, slice) + fa.sharedSizeBytes <= (size_t)smem_optin;
    const void* fn = in_smem ? (const void*)pcg_cluster_kernel<true> : (const void*)pcg_cluster_kernel<false>;
    const size_t smem = cluster_smem(rows, in_smem ? slice : -1);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
    e = cudaOccupancyMaxActiveClusters(&active, fn, &cfg);
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
    P.timeout_ns = (uint64_t)(h->timeout_ms * 1e6);
    P.skip_seq = h->skip_seq;
    P.st = h->st;
    if ((e = cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream)) != cudaSuccess) return cuda_err(e, "memset");
    if ((e = cudaEventRecord(h->ev0, h->stream)) != cudaSuccess) return cuda_err(e, "event");
    e = in_smem ? cudaLaunchKernelEx(&cfg, pcg_cluster_kernel<true>, P)
                : cudaLaunchKernelEx(&cfg, pcg_cluster_kernel<false>, P);
    if (e != cudaSuccess) return cuda_err(e, "launch");
    if ((e = cudaEventRecord(h->ev1, h->stream)) != cudaSuccess) return cuda_err(e, "event");
    if ((e = cudaMemcpyAsync(h->host_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
      return cuda_err(e, "status copy");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_err(e, "synchronize");
    csr_in_smem = in_smem;
    break;
  }
  float ms = 0.0f;
  if ((e = cudaEventElapsedTime(&ms, h->ev0, h->ev1)) != cudaSuccess) return cuda_err(e, "event time");
  const DevState& ds = *h->host_st;
  const cg_status status = ds.abort ? CG_ERR_TIMEOUT : (cg_status)ds.status;
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
  // bytes the loop reads from outside the SMs per iteration: none with the CSR in
  // shared memory, else the CSR from L1/L2 (the vectors stay on chip either way)
  h->last.kernel_bytes_per_iter = csr_in_smem ? 0 : 12 * nnz + 4 * (n + 1);
  if (iters_out) *iters_out = ds.iters;
  if (relres_out) *relres_out = ds.relres_true;
  if (status == CG_ERR_TIMEOUT) {
    h->err = "cg_solve (cluster form): a bounded wait gave up (exchange " + std::to_string(ds.err_barrier) +
             ", CTA " + std::to_string(ds.err_cta) + "); timed out";
  } else if (status < 0) {
    h->err = std::string("cg_solve: ") + cg_status_string(status);
  }
  return status;
}
