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
#include "cg_graph.cuh"
#include "cg_fsai.cuh"

using namespace cg;

namespace {

thread_local std::string g_create_error;

}  // namespace

void cgi::set_create_error(const std::string& msg) { g_create_error = msg; }

namespace {

// Device checks of a CSR whose rowptr the host has already validated:
// colind in [0, n); per row the diagonal sum A_ii and the number of stored
// diagonal entries; counters[1] counts rows without a positive diagonal.
__global__ void validate_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ colind, const double* __restrict__ vals,
                                double* diag, int32_t* ndiag, unsigned long long* counters) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int a = rowptr[i], e = rowptr[i + 1];
    double d = 0.0;
    int found = 0;
    unsigned long long bad = 0;
    for (int k = a; k < e; ++k) {
      const int c = colind[k];
      if (c < 0 || (int64_t)c >= n) { ++bad; continue; }
      if ((int64_t)c == i) { d += vals[k]; ++found; }
    }
    if (bad) atomicAdd(&counters[0], bad);
    diag[i] = d;
    ndiag[i] = found;
    if (!(found && d > 0.0)) atomicAdd(&counters[1], 1ull);
  }
}

// Diagonal vectors: sqrt(A_ii), 1/sqrt(A_ii) (Jacobi scaling) and fp32 copies.
__global__ void diag_kernel(int64_t n, const double* __restrict__ diag, double* dsq, double* disq,
                            float* diag32, float* disq32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = diag[i];
    const double s = d > 0.0 ? sqrt(d) : 0.0;
    const double si = d > 0.0 ? 1.0 / s : 0.0;
    dsq[i] = s;
    disq[i] = si;
    diag32[i] = (float)d;
    disq32[i] = (float)si;
  }
}

// SELL-32 slices of the off-diagonal part (thread per row i): entries of a
// short row go to column m of its slice in storage order, the rest of the
// slice width is padding (column = i, value = 0); a long row (more than
// kLongRow off-diagonal entries) gets padding only.  With SCALE the values
// become A_ij / sqrt(A_ii A_jj) (the product of the two scales is formed
// first, so A^ stays bitwise symmetric when A is).  col may be null (already
// written by an earlier value variant).
template <typename T, bool SCALE>
__global__ void fill_sell_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colind,
                                 const double* __restrict__ vals,
                                 const int32_t* __restrict__ ndiag,
                                 const double* __restrict__ disq,
                                 const int32_t* __restrict__ soff, const int32_t* __restrict__ spos,
                                 int32_t* col, T* val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ps = spos ? (int64_t)spos[i] : i;  // slice position of row i
    const int64_t s = ps >> 5, l = ps & 31;
    const int64_t base = (int64_t)soff[s] * 32 + l;
    const int w = soff[s + 1] - soff[s];
    const int len = rowptr[i + 1] - rowptr[i] - ndiag[i];
    int m = 0;
    if (len <= kLongRow) {
      const double si = SCALE ? disq[i] : 1.0;
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int c = colind[k];
        if ((int64_t)c == i) continue;
        if (col) col[base + (int64_t)m * 32] = c;
        val[base + (int64_t)m * 32] = (T)(SCALE ? vals[k] * (si * disq[c]) : vals[k]);
        ++m;
      }
    }
    for (; m < w; ++m) {
      if (col) col[base + (int64_t)m * 32] = (int32_t)i;
      val[base + (int64_t)m * 32] = T(0);
    }
  }
}

// The CSR loop layout (thread per row): row i's off-diagonal entries in
// storage order at [lrp[ps], lrp[ps+1]), ps = spos[i] its position; with
// SCALE the Jacobi scaling as above.
template <typename T, bool SCALE>
__global__ void fill_csr_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                const double* __restrict__ vals, const double* __restrict__ disq,
                                const int32_t* __restrict__ lrp, const int32_t* __restrict__ spos, int32_t* col,
                                T* val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = lrp[spos[i]];
    const double si = SCALE ? disq[i] : 1.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int c = colind[k];
      if ((int64_t)c == i) continue;
      if (col) col[o] = c;
      val[o] = (T)(SCALE ? vals[k] * (si * disq[c]) : vals[k]);
      ++o;
    }
  }
}

// Range of a positive diagonal: min / max of the IEEE bit patterns, which
// order like the values for positive doubles.
__global__ void diag_range_kernel(int64_t n, const double* __restrict__ d, unsigned long long* mm) {
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d[i]);
    lo = b < lo ? b : lo;
    hi = b > hi ? b : hi;
  }
  atomicMin(&mm[0], lo);
  atomicMax(&mm[1], hi);
}

// Distinct off-diagonal offsets j - i into a 64-slot open-addressing table
// (kOffEmpty marks a free slot); *overflow is set when they do not fit.
constexpr int kOffSlots = 64;
constexpr int kOffEmpty = INT32_MIN;
__global__ void offsets_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                               const int32_t* __restrict__ colind, int* table, int* overflow) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int64_t c = colind[k];
      if (c == i) continue;
      const int d = (int)(c - i);
      unsigned h = ((unsigned)d * 2654435761u) >> 26;  // 6 bits
      int t = 0;
      for (; t < kOffSlots; ++t, h = (h + 1) & (kOffSlots - 1)) {
        const int v = *((volatile int*)&table[h]);
        if (v == d) break;
        if (v == kOffEmpty) {
          const int old = atomicCAS(&table[h], kOffEmpty, d);
          if (old == kOffEmpty || old == d) break;
        }
      }
      if (t == kOffSlots) atomicExch(overflow, 1);
    }
  }
}

// Sliced-diagonal values (thread per row): slot m of row i holds the sum of
// the row's entries in column i + delta[m] (0 where there is none); with
// SCALE the Jacobi scaling A_ij / sqrt(A_ii A_jj).  The array is zeroed
// before, so lanes past n stay 0.
template <typename T, bool SCALE>
__global__ void fill_dia_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ colind,
                                const double* __restrict__ vals,
                                const double* __restrict__ disq, int ndiag,
                                const int32_t* __restrict__ delta, T* val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = (i >> 5) * ndiag * 32 + (i & 31);
    const double si = SCALE ? disq[i] : 1.0;
    for (int m = 0; m < ndiag; ++m) {
      const int64_t target = i + delta[m];
      double v = 0.0;
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
        if ((int64_t)colind[k] == target) v += SCALE ? vals[k] * (si * disq[target]) : vals[k];
      val[base + (int64_t)m * 32] = (T)v;
    }
  }
}

// Compact CSR of the long rows (thread per long row).
template <typename T, bool SCALE>
__global__ void fill_long_kernel(int32_t nlong, const int32_t* __restrict__ lrow,
                                 const int32_t* __restrict__ lptr,
                                 const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colind,
                                 const double* __restrict__ vals,
                                 const double* __restrict__ disq, int32_t* lcol, T* lval) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nlong;
       l += (int64_t)gridDim.x * blockDim.x) {
    const int i = lrow[l];
    int ko = lptr[l];
    const double si = SCALE ? disq[i] : 1.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int c = colind[k];
      if (c == i) continue;
      if (lcol) lcol[ko] = c;
      lval[ko] = (T)(SCALE ? vals[k] * (si * disq[c]) : vals[k]);
      ++ko;
    }
  }
}

}  // namespace

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

unsigned grid_for(int64_t items) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 65535));
}

// Cut rows into row blocks: greedily extend a block while it stays within
// kCapV nonzeros and kBlock rows; a row longer than kCapV gets a block alone.
std::vector<int32_t> build_row_blocks(const int32_t* rowptr, int64_t n, int64_t* long_rows) {
  std::vector<int32_t> rb;
  rb.reserve((size_t)(n / 64 + 2));
  rb.push_back(0);
  int64_t r = 0, longs = 0;
  while (r < n) {
    const int64_t start = r;
    const int64_t len0 = rowptr[r + 1] - rowptr[r];
    if (len0 > kCapV) {
      ++r;
      ++longs;
    } else {
      int64_t nk = 0;
      while (r < n && r - start < kBlock) {
        const int64_t len = rowptr[r + 1] - rowptr[r];
        if (nk + len > kCapV) break;
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

// Loop-matrix bytes beyond the entries read once per SpMV: the row of each
// slice position (SELL-C-sigma) or the row pointers (CSR layout).
int64_t loop_index_bytes(const cg_handle* h) {
  return (h->sperm ? 4 * h->n : 0) + (h->csr ? 4 * (h->n + 1) : 0);
}

// The caller's CSR for the SpMV kernels; 16-byte loads when both arrays allow them.
Csr<double> make_csr(const cg_handle* h) {
  return Csr<double>{h->n, h->rowptr, h->colind, h->vals, h->rb, h->nrb,
                     (aligned16(h->colind) && aligned16(h->vals)) ? 1 : 0};
}

// Grid of the stand-alone caller-CSR SpMV: every resident CTA, each taking row
// blocks round-robin.
unsigned spmv_grid(const cg_handle* h) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmv_kernel<double>, kBlock, 0) != cudaSuccess ||
      per_sm <= 0)
    per_sm = 4;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(h->nrb, (int64_t)per_sm * h->sm_count));
}

int auto_grid(const cg_handle* h) {
  if (h->grid_opt > 0) return std::min(h->grid_opt, h->grid_max);
  // enough CTAs for the larger of the row-block and vector work, capped by residency
  const int64_t vec_ctas = (h->n / 2 + kBlock - 1) / kBlock;
  const int64_t want = std::max<int64_t>(1, std::max<int64_t>(h->nrb, vec_ctas));
  return (int)std::min<int64_t>(want, h->grid_max);
}

}  // namespace

// Every distinct off-diagonal offset j - i of the caller's CSR, once per
// handle (device table of kOffSlots slots; noffs_all = -1 when they do not fit).
cg_status cgi::ensure_offsets(cg_handle* h) {
  if (h->noffs_all != cg_handle::kOffsUnknown) return CG_OK;
  const int64_t n = h->n;
  std::vector<int> ht(kOffSlots + 1, kOffEmpty);
  ht[kOffSlots] = 0;
  if (n > 0) {
    int* tab = nullptr;
    CG_CUDA(h, cudaMalloc(&tab, sizeof(int) * (kOffSlots + 1)));
    cudaError_t e = cudaMemcpy(tab, ht.data(), sizeof(int) * (kOffSlots + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      offsets_kernel<<<grid_for(n), 256>>>(n, h->rowptr, h->colind, tab, tab + kOffSlots);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(ht.data(), tab, sizeof(int) * (kOffSlots + 1), cudaMemcpyDeviceToHost);
    cudaFree(tab);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagonal offsets");
  }
  std::vector<int32_t> offs;
  for (int t = 0; t < kOffSlots; ++t)
    if (ht[(size_t)t] != kOffEmpty) offs.push_back(ht[(size_t)t]);
  std::sort(offs.begin(), offs.end());
  static_assert(kOffSlots <= cg_handle::kOffsAll, "offset table larger than the handle's copy");
  h->noffs_all = ht[kOffSlots] ? -1 : (int32_t)offs.size();
  for (int m = 0; m < std::max(h->noffs_all, 0); ++m) h->offs_all[m] = offs[(size_t)m];
  return CG_OK;
}

namespace {

// SELL-32 structure of the off-diagonal part (shared by every value
// variant) and the diagonal vectors.
cg_status ensure_offdiag(cg_handle* h) {
  if (h->soff) return CG_OK;
  const int64_t n = h->n;
  std::vector<int32_t> nd((size_t)n);
  if (n > 0) CG_CUDA(h, cudaMemcpy(nd.data(), h->ndiag, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost));
  const std::vector<int32_t>& rp = h->host_rowptr;
  const int64_t ns = (n + 31) / 32;
  // sliced-diagonal layout when the off-diagonal part lies on <= kMaxDiag
  // diagonals that are at least 90 % full
  int64_t nnz_od_all = 0;
  for (int64_t i = 0; i < n; ++i) nnz_od_all += rp[(size_t)i + 1] - rp[(size_t)i] - nd[(size_t)i];
  if (n > 0 && nnz_od_all > 0) {
    const cg_status so = cgi::ensure_offsets(h);
    if (so != CG_OK) return so;
    const int nd_ = std::max(h->noffs_all, 0);
    const bool fits = h->noffs_all >= 0;
    std::vector<int32_t> offs(h->offs_all, h->offs_all + nd_);
    if (fits && nd_ > 0 && nd_ <= kMaxDiag && nnz_od_all * 10 >= (int64_t)nd_ * n * 9) {
      h->dia = 1;
      h->uniform_w = nd_;
      for (int m = 0; m < nd_; ++m) h->delta[m] = offs[(size_t)m];
      h->nslices = (int32_t)ns;
      h->sell_entries = ns * 32 * nd_;
      h->nnz_od = nnz_od_all;
      h->nlong = 0;
      h->nnz_long = 0;
      std::vector<int32_t> soff((size_t)ns + 1);
      for (int64_t s2 = 0; s2 <= ns; ++s2) soff[(size_t)s2] = (int32_t)(s2 * nd_);
      std::vector<uint32_t> lmask((size_t)std::max<int64_t>(ns, 1), 0u);
      CG_CUDA(h, cudaMalloc(&h->soff, sizeof(int32_t) * soff.size()));
      CG_CUDA(h, cudaMemcpy(h->soff, soff.data(), sizeof(int32_t) * soff.size(), cudaMemcpyHostToDevice));
      CG_CUDA(h, cudaMalloc(&h->lmask, sizeof(uint32_t) * lmask.size()));
      CG_CUDA(h, cudaMemcpy(h->lmask, lmask.data(), sizeof(uint32_t) * lmask.size(), cudaMemcpyHostToDevice));
      CG_CUDA(h, cudaMalloc(&h->delta_dev, sizeof(int32_t) * kMaxDiag));
      CG_CUDA(h, cudaMemcpy(h->delta_dev, h->delta, sizeof(int32_t) * kMaxDiag, cudaMemcpyHostToDevice));
      CG_CUDA(h, cudaMalloc(&h->lptr, sizeof(int32_t)));
      CG_CUDA(h, cudaMemset(h->lptr, 0, sizeof(int32_t)));
      const size_t nv = (size_t)std::max<int64_t>(n, 1);
      CG_CUDA(h, cudaMalloc(&h->dsq, sizeof(double) * nv));
      CG_CUDA(h, cudaMalloc(&h->disq, sizeof(double) * nv));
      CG_CUDA(h, cudaMalloc(&h->diag32, sizeof(float) * nv));
      CG_CUDA(h, cudaMalloc(&h->disq32, sizeof(float) * nv));
      diag_kernel<<<grid_for(n), 256>>>(n, h->diag, h->dsq, h->disq, h->diag32, h->disq32);
      CG_CUDA(h, cudaGetLastError());
      CG_CUDA(h, cudaDeviceSynchronize());
      return CG_OK;
    }
  }
  std::vector<int32_t> soff((size_t)ns + 1, 0);
  std::vector<uint32_t> lmask((size_t)std::max<int64_t>(ns, 1), 0u);
  std::vector<int32_t> lrow, lptr(1, 0);
  std::vector<int32_t> width((size_t)std::max<int64_t>(ns, 1), 0);
  std::vector<int32_t> slen((size_t)std::max<int64_t>(n, 1), 0);  // slice length of each row (0: long)
  int64_t sumw = 0, nnz_od = 0;
  int maxw = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int len = rp[(size_t)i + 1] - rp[(size_t)i] - nd[(size_t)i];
    nnz_od += len;
    if (len > kLongRow) {
      lrow.push_back((int32_t)i);
      lptr.push_back(lptr.back() + len);
    } else {
      slen[(size_t)i] = len;
    }
  }
  for (int64_t s = 0; s < ns; ++s) {
    int w = 0;
    for (int64_t i = s * 32; i < std::min<int64_t>(n, s * 32 + 32); ++i) w = std::max(w, slen[(size_t)i]);
    width[(size_t)s] = w;
    sumw += w;
    maxw = std::max(maxw, w);
  }
  // uniform slices (offsets computed, not loaded) when that pads by <= 1/16
  const bool uniform = lrow.empty() && ns > 0 && (int64_t)maxw * ns * 16 <= sumw * 17;
  std::vector<int32_t> perm, spos;
  if (!uniform && n > 0) {
    // SELL-C-sigma: within each window of kSellSigma rows, rows sorted by
    // descending slice length (stable), so a slice's rows have similar lengths
    perm.assign((size_t)ns * 32, (int32_t)n);  // dead positions: n
    spos.assign((size_t)n, 0);
    std::vector<int32_t> idx;
    for (int64_t r0 = 0; r0 < n; r0 += kSellSigma) {
      const int64_t r1 = std::min<int64_t>(n, r0 + kSellSigma);
      idx.resize((size_t)(r1 - r0));
      for (int64_t i = r0; i < r1; ++i) idx[(size_t)(i - r0)] = (int32_t)i;
      std::stable_sort(idx.begin(), idx.end(),
                       [&](int32_t a, int32_t b) { return slen[(size_t)a] > slen[(size_t)b]; });
      for (int64_t k = 0; k < r1 - r0; ++k) {
        perm[(size_t)(r0 + k)] = idx[(size_t)k];
        spos[(size_t)idx[(size_t)k]] = (int32_t)(r0 + k);
      }
    }
    sumw = 0;
    for (int64_t s = 0; s < ns; ++s) {
      int w = 0;
      for (int64_t ps = s * 32; ps < s * 32 + 32; ++ps) {
        const int32_t i = perm[(size_t)ps];
        if (i >= n) continue;
        w = std::max(w, slen[(size_t)i]);
        const int len = rp[(size_t)i + 1] - rp[(size_t)i] - nd[(size_t)i];
        if (len > kLongRow) lmask[(size_t)s] |= 1u << (ps & 31);
      }
      width[(size_t)s] = w;
      sumw += w;
    }
  } else {
    for (int64_t s = 0; s < ns; ++s)
      for (int64_t i = s * 32; i < std::min<int64_t>(n, s * 32 + 32); ++i) {
        const int len = rp[(size_t)i + 1] - rp[(size_t)i] - nd[(size_t)i];
        if (len > kLongRow) lmask[(size_t)s] |= 1u << (i & 31);
      }
  }
  h->uniform_w = uniform ? maxw : -1;
  // rows too uneven for slices even after sorting (a heavy tail of row
  // lengths): the loop matrix becomes a CSR of the off-diagonal entries in row
  // blocks, summed by the binned row-block kernel
  if (!uniform && n > 0 && 32 * sumw > (int64_t)(kCsrPadLimit * (double)std::max<int64_t>(1, nnz_od - lptr.back()))) {
    std::vector<int32_t> lrp((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i)
      lrp[(size_t)i + 1] = lrp[(size_t)i] + (rp[(size_t)i + 1] - rp[(size_t)i] - nd[(size_t)i]);
    int64_t longs = 0;
    std::vector<int32_t> lrb = build_row_blocks(lrp.data(), n, &longs);
    // within each row block the rows go in order of descending length (stable):
    // a warp's rows then have similar lengths, and its fp64 FMAs, which GB300
    // issues per warp whatever the active lanes, run only to its longest row.
    // Blocks keep their rows and entries, so their boundaries are unchanged;
    // perm maps a position to its row, spos a row to its position.
    perm.assign((size_t)n, 0);
    spos.assign((size_t)n, 0);
    {
      std::vector<int32_t> idx;
      for (size_t b = 0; b + 1 < lrb.size(); ++b) {
        const int64_t r0 = lrb[b], r1 = lrb[b + 1];
        idx.resize((size_t)(r1 - r0));
        for (int64_t i = r0; i < r1; ++i) idx[(size_t)(i - r0)] = (int32_t)i;
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
          return lrp[(size_t)x + 1] - lrp[(size_t)x] > lrp[(size_t)y + 1] - lrp[(size_t)y];
        });
        for (int64_t k = 0; k < r1 - r0; ++k) {
          perm[(size_t)(r0 + k)] = idx[(size_t)k];
          spos[(size_t)idx[(size_t)k]] = (int32_t)(r0 + k);
        }
      }
      std::vector<int32_t> prp((size_t)n + 1, 0);
      for (int64_t ps = 0; ps < n; ++ps) {
        const int32_t i = perm[(size_t)ps];
        prp[(size_t)ps + 1] = prp[(size_t)ps] + (lrp[(size_t)i + 1] - lrp[(size_t)i]);
      }
      lrp.swap(prp);
    }
    CG_CUDA(h, cudaMalloc(&h->sperm, sizeof(int32_t) * perm.size()));
    CG_CUDA(h, cudaMemcpy(h->sperm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice));
    CG_CUDA(h, cudaMalloc(&h->spos, sizeof(int32_t) * spos.size()));
    CG_CUDA(h, cudaMemcpy(h->spos, spos.data(), sizeof(int32_t) * spos.size(), cudaMemcpyHostToDevice));
    h->csr = 1;
    h->uniform_w = -1;
    h->nslices = 0;
    h->sell_entries = nnz_od;
    h->nnz_od = nnz_od;
    h->nlong = 0;
    h->nnz_long = 0;
    h->lnrb = (int32_t)(lrb.size() - 1);
    const size_t nv = (size_t)std::max<int64_t>(n, 1);
    CG_CUDA(h, cudaMalloc(&h->lrp, sizeof(int32_t) * lrp.size()));
    CG_CUDA(h, cudaMemcpy(h->lrp, lrp.data(), sizeof(int32_t) * lrp.size(), cudaMemcpyHostToDevice));
    CG_CUDA(h, cudaMalloc(&h->lrb, sizeof(int32_t) * lrb.size()));
    CG_CUDA(h, cudaMemcpy(h->lrb, lrb.data(), sizeof(int32_t) * lrb.size(), cudaMemcpyHostToDevice));
    CG_CUDA(h, cudaMalloc(&h->scol, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz_od, 4)));
    CG_CUDA(h, cudaMalloc(&h->soff, sizeof(int32_t)));
    CG_CUDA(h, cudaMalloc(&h->lmask, sizeof(uint32_t)));
    CG_CUDA(h, cudaMalloc(&h->lrow, sizeof(int32_t)));
    CG_CUDA(h, cudaMalloc(&h->lptr, sizeof(int32_t)));
    CG_CUDA(h, cudaMemset(h->lptr, 0, sizeof(int32_t)));
    CG_CUDA(h, cudaMalloc(&h->lcol, sizeof(int32_t)));
    CG_CUDA(h, cudaMalloc(&h->dsq, sizeof(double) * nv));
    CG_CUDA(h, cudaMalloc(&h->disq, sizeof(double) * nv));
    CG_CUDA(h, cudaMalloc(&h->diag32, sizeof(float) * nv));
    CG_CUDA(h, cudaMalloc(&h->disq32, sizeof(float) * nv));
    diag_kernel<<<grid_for(n), 256>>>(n, h->diag, h->dsq, h->disq, h->diag32, h->disq32);
    CG_CUDA(h, cudaGetLastError());
    CG_CUDA(h, cudaDeviceSynchronize());
    return CG_OK;
  }
  int64_t off = 0;
  for (int64_t s = 0; s < ns; ++s) {
    off += uniform ? maxw : width[(size_t)s];
    if (off >= INT32_MAX / 32) return fail(h, CG_ERR_INVALID, "cg_create: padded matrix too large");
    soff[(size_t)s + 1] = (int32_t)off;
  }
  if (!perm.empty()) {
    CG_CUDA(h, cudaMalloc(&h->sperm, sizeof(int32_t) * perm.size()));
    CG_CUDA(h, cudaMemcpy(h->sperm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice));
    CG_CUDA(h, cudaMalloc(&h->spos, sizeof(int32_t) * spos.size()));
    CG_CUDA(h, cudaMemcpy(h->spos, spos.data(), sizeof(int32_t) * spos.size(), cudaMemcpyHostToDevice));
  }
  h->nslices = (int32_t)ns;
  h->sell_entries = off * 32;
  h->nnz_od = nnz_od;
  h->nlong = (int32_t)lrow.size();
  h->nnz_long = lptr.back();
  const size_t nv = (size_t)std::max<int64_t>(n, 1);
  CG_CUDA(h, cudaMalloc(&h->soff, sizeof(int32_t) * soff.size()));
  CG_CUDA(h, cudaMemcpy(h->soff, soff.data(), sizeof(int32_t) * soff.size(), cudaMemcpyHostToDevice));
  CG_CUDA(h, cudaMalloc(&h->lmask, sizeof(uint32_t) * lmask.size()));
  CG_CUDA(h, cudaMemcpy(h->lmask, lmask.data(), sizeof(uint32_t) * lmask.size(), cudaMemcpyHostToDevice));
  CG_CUDA(h, cudaMalloc(&h->scol, sizeof(int32_t) * (size_t)std::max<int64_t>(h->sell_entries, 1)));
  // lanes without a row (past n, or dead SELL-C-sigma positions) are never filled:
  // column 0 and value 0 keep their loads in bounds and their products zero
  CG_CUDA(h, cudaMemset(h->scol, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(h->sell_entries, 1)));
  CG_CUDA(h, cudaMalloc(&h->lrow, sizeof(int32_t) * std::max<size_t>(lrow.size(), 1)));
  CG_CUDA(h, cudaMalloc(&h->lptr, sizeof(int32_t) * lptr.size()));
  CG_CUDA(h, cudaMalloc(&h->lcol, sizeof(int32_t) * (size_t)std::max<int64_t>(h->nnz_long, 1)));
  if (!lrow.empty())
    CG_CUDA(h, cudaMemcpy(h->lrow, lrow.data(), sizeof(int32_t) * lrow.size(), cudaMemcpyHostToDevice));
  CG_CUDA(h, cudaMemcpy(h->lptr, lptr.data(), sizeof(int32_t) * lptr.size(), cudaMemcpyHostToDevice));
  CG_CUDA(h, cudaMalloc(&h->dsq, sizeof(double) * nv));
  CG_CUDA(h, cudaMalloc(&h->disq, sizeof(double) * nv));
  CG_CUDA(h, cudaMalloc(&h->diag32, sizeof(float) * nv));
  CG_CUDA(h, cudaMalloc(&h->disq32, sizeof(float) * nv));
  if (n > 0) {
    diag_kernel<<<grid_for(n), 256>>>(n, h->diag, h->dsq, h->disq, h->diag32, h->disq32);
    CG_CUDA(h, cudaGetLastError());
    CG_CUDA(h, cudaDeviceSynchronize());
  }
  return CG_OK;
}

// Loop-matrix values for (precision, precond), built on first use; the first
// variant built also writes the shared column indices.
template <typename T>
cg_status ensure_vals(cg_handle* h, T** sval, T** lval, bool scale) {
  if (*sval) return CG_OK;
  cg_status s = ensure_offdiag(h);
  if (s != CG_OK) return s;
  const bool write_col = !h->scol_written;
  CG_CUDA(h, cudaMalloc(sval, sizeof(T) * (size_t)std::max<int64_t>(h->sell_entries, 1)));
  CG_CUDA(h, cudaMalloc(lval, sizeof(T) * (size_t)std::max<int64_t>(h->nnz_long, 1)));
  if (h->csr) {
    if (h->n > 0) {
      if (scale)
        fill_csr_kernel<T, true><<<grid_for(h->n), 256>>>(h->n, h->rowptr, h->colind, h->vals, h->disq, h->lrp,
                                                          h->spos, write_col ? h->scol : nullptr, *sval);
      else
        fill_csr_kernel<T, false><<<grid_for(h->n), 256>>>(h->n, h->rowptr, h->colind, h->vals, h->disq, h->lrp,
                                                           h->spos, write_col ? h->scol : nullptr, *sval);
      CG_CUDA(h, cudaGetLastError());
      CG_CUDA(h, cudaDeviceSynchronize());
    }
    h->scol_written = true;
    return CG_OK;
  }
  if (h->dia) {
    CG_CUDA(h, cudaMemset(*sval, 0, sizeof(T) * (size_t)std::max<int64_t>(h->sell_entries, 1)));
    if (scale)
      fill_dia_kernel<T, true><<<grid_for(h->n), 256>>>(h->n, h->rowptr, h->colind, h->vals, h->disq,
                                                        h->uniform_w, h->delta_dev, *sval);
    else
      fill_dia_kernel<T, false><<<grid_for(h->n), 256>>>(h->n, h->rowptr, h->colind, h->vals, h->disq,
                                                         h->uniform_w, h->delta_dev, *sval);
    CG_CUDA(h, cudaGetLastError());
    CG_CUDA(h, cudaDeviceSynchronize());
    return CG_OK;
  }
  CG_CUDA(h, cudaMemset(*sval, 0, sizeof(T) * (size_t)std::max<int64_t>(h->sell_entries, 1)));
  if (h->n > 0) {
    int32_t* col = write_col ? h->scol : nullptr;
    int32_t* lcol = write_col ? h->lcol : nullptr;
    if (scale) {
      fill_sell_kernel<T, true><<<grid_for(h->n), 256>>>(h->n, h->rowptr, h->colind, h->vals,
                                                         h->ndiag, h->disq, h->soff, h->spos, col, *sval);
      if (h->nlong)
        fill_long_kernel<T, true><<<grid_for(h->nlong), 256>>>(h->nlong, h->lrow, h->lptr,
                                                               h->rowptr, h->colind, h->vals,
                                                               h->disq, lcol, *lval);
    } else {
      fill_sell_kernel<T, false><<<grid_for(h->n), 256>>>(h->n, h->rowptr, h->colind, h->vals,
                                                          h->ndiag, h->disq, h->soff, h->spos, col, *sval);
      if (h->nlong)
        fill_long_kernel<T, false><<<grid_for(h->nlong), 256>>>(h->nlong, h->lrow, h->lptr,
                                                                h->rowptr, h->colind, h->vals,
                                                                h->disq, lcol, *lval);
    }
    CG_CUDA(h, cudaGetLastError());
    CG_CUDA(h, cudaDeviceSynchronize());
  }
  h->scol_written = true;
  return CG_OK;
}

template <typename T>
Sell<T> make_sell(const cg_handle* h, const T* val, const T* lval, const T* diag, const T* disq) {
  Sell<T> S{};
  S.n = h->n;
  S.nslices = h->nslices;
  S.uw = h->uniform_w;
  S.dia = h->dia;
  for (int m = 0; m < kMaxDiag; ++m) S.delta[m] = h->delta[m];
  S.soff = h->soff;
  S.perm = h->sperm;
  S.csr = h->csr;
  S.nrb = h->lnrb;
  S.rptr = h->lrp;
  S.rb = h->lrb;
  S.lmask = h->lmask;
  S.col = h->scol;
  S.val = val;
  S.nlong = h->nlong;
  S.lrow = h->lrow;
  S.lptr = h->lptr;
  S.lcol = h->lcol;
  S.lval = lval;
  S.dg = diag;
  S.dn = diag;
  S.disq = disq;
  S.dmin = h->dmin;
  S.dmax = h->dmax;
  return S;
}

template <typename T>
cg_status ensure_vectors(cg_handle* h, T** r, T** p, T** q, T** xh) {
  if (*r) return CG_OK;
  const size_t nv = (size_t)std::max<int64_t>(h->n, 1);
  CG_CUDA(h, cudaMalloc(r, sizeof(T) * nv));
  CG_CUDA(h, cudaMalloc(p, sizeof(T) * nv));
  CG_CUDA(h, cudaMalloc(q, sizeof(T) * nv));
  CG_CUDA(h, cudaMalloc(xh, sizeof(T) * nv));
  return CG_OK;
}

void destroy_graph(cudaGraphExec_t* e, cudaGraph_t* g) {
  if (*e) { cudaGraphExecDestroy(*e); *e = nullptr; }
  if (*g) { cudaGraphDestroy(*g); *g = nullptr; }
}

void free_all(cg_handle* h) {
  if (h->batch) cgi::batch_free(h->batch);
  if (h->fsai) cgi::fsai_free(h->fsai);
  void* dev[] = {h->rb,        h->diag,      h->ndiag,     h->dsq,       h->disq,       h->delta_dev,
                 h->diag32,    h->disq32,    h->soff,      h->lmask,     h->scol,
                 h->lrow,      h->lptr,      h->lcol,      h->sval64[0], h->sval64[1],
                 h->sval32[0], h->sval32[1], h->lval64[0], h->lval64[1], h->lval32[0],
                 h->lval32[1], h->r,         h->p,         h->q,         h->xh,
                 h->r32,       h->p32,       h->q32,       h->xh32,      h->part,
                 h->st,        h->stage_b,   h->stage_x,   h->sperm,     h->spos,
                 h->lrp,       h->lrb};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (h->host_st) cudaFreeHost(h->host_st);
  if (h->host_gs) cudaFreeHost(h->host_gs);
  if (h->gs) cudaFree(h->gs);
  destroy_graph(&h->gexec, &h->graph);
  destroy_graph(&h->gexec_it, &h->graph_it);
  destroy_graph(&h->gexec_ep, &h->graph_ep);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
}

// The graph-mode SpMV kernel for the loop matrix's slice layout.
template <typename T, bool JAC, bool DIA>
const void* spmv_kernel_w(int uw) {
  switch (uw) {
    case 4: return (const void*)g_spmv<T, JAC, 4, DIA>;
    case 6: return (const void*)g_spmv<T, JAC, 6, DIA>;
    case 8: return (const void*)g_spmv<T, JAC, 8, DIA>;
    case 26: return DIA ? (const void*)g_spmv_wide<T, JAC, 26, true> : (const void*)g_spmv_gen<T, JAC>;
    default: return (const void*)g_spmv_gen<T, JAC>;
  }
}
template <typename T>
const void* spmv_kernel_for(int uw, bool dia, bool jac, bool csr = false) {
  if (csr) return jac ? (const void*)g_spmv_csr<T, true> : (const void*)g_spmv_csr<T, false>;
  if (jac) return dia ? spmv_kernel_w<T, true, true>(uw) : spmv_kernel_w<T, true, false>(uw);
  return dia ? spmv_kernel_w<T, false, true>(uw) : spmv_kernel_w<T, false, false>(uw);
}

}  // namespace

namespace {

// Append a kernel node after `dep` (may be null) to graph g.
template <typename... Args>
cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, cudaGraphNode_t dep, const void* fn,
                       unsigned grid, unsigned block, void** args) {
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
}

// Build and instantiate the graph form of an fp64 solve for (b, x, tol, maxit,
// precond).  unroll == 0: one graph [prologue, WHILE{3 phase kernels},
// epilogue].  unroll > 0: three graphs (prologue, `unroll` iterations whose
// kernels return at once after the loop has stopped, epilogue) that the host
// launches in turn, reading the loop state after each iteration graph.
cg_status build_graph64(cg_handle* h, const SolveParams& P, bool jac, int unroll) {
  destroy_graph(&h->gexec, &h->graph);
  destroy_graph(&h->gexec_it, &h->graph_it);
  destroy_graph(&h->gexec_ep, &h->graph_ep);
  cudaGraph_t g;
  CG_CUDA(h, cudaGraphCreate(&g, 0));
  h->graph = g;
  cudaGraphConditionalHandle ch = 0;
  if (unroll == 0) CG_CUDA(h, cudaGraphConditionalHandleCreate(&ch, g, 0, cudaGraphCondAssignDefault));
  const void* f_spmv = spmv_kernel_for<double>(h->uniform_w, h->dia != 0, jac, h->csr != 0);
  const unsigned G = (unsigned)h->grid_graph;
  const unsigned Gq = (unsigned)std::max(1, std::min(max_coresident(f_spmv, h->sm_count),
                                                     h->grid_part));
  GArgs ga{P, h->gs, ch, 0, Gq, G};
  Csr<double> A = P.A;
  const double* x = P.x;
  double* q = P.V64.q;
  const unsigned Gs = spmv_grid(h);
  void* a_spmv[] = {&A, &x, &q};
  void* a_ga[] = {&ga};
  const void* f_r = jac ? (const void*)g_upd_r<double, true> : (const void*)g_upd_r<double, false>;
  const void* f_xp =
      unroll == 0 ? (jac ? (const void*)g_upd_xp<double, true, false, true>
                         : (const void*)g_upd_xp<double, false, false, true>)
                  : (jac ? (const void*)g_upd_xp<double, true, false, false>
                         : (const void*)g_upd_xp<double, false, false, false>);
  const void* f_flush = jac ? (const void*)g_flush<double, true, false>
                            : (const void*)g_flush<double, false, false>;
  const bool with_rr = jac && h->dmin != h->dmax;  // r.r fallback kernel needed
  cudaGraphNode_t n, prev;
  // prologue
  CG_CUDA(h, add_kernel(g, &n, nullptr, (const void*)spmv_kernel<double>, Gs, kBlock, a_spmv));
  prev = n;
  CG_CUDA(h, add_kernel(g, &n, prev, jac ? (const void*)g_res64<true> : (const void*)g_res64<false>,
                        G, kBlock, a_ga));
  prev = n;
  CG_CUDA(h, add_kernel(g, &n, prev,
                        unroll == 0 ? (const void*)g_start64<true> : (const void*)g_start64<false>,
                        1, 32, a_ga));
  prev = n;
  cudaGraph_t ep = g;
  if (unroll == 0) {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = ch;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CG_CUDA(h, cudaGraphAddNode(&n, g, &prev, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphNode_t b1, b2, b3;
    CG_CUDA(h, add_kernel(body, &b1, nullptr, f_spmv, Gq, kBlock, a_ga));
    CG_CUDA(h, add_kernel(body, &b2, b1, f_r, G, kBlock, a_ga));
    if (with_rr) {
      CG_CUDA(h, add_kernel(body, &b3, b2, (const void*)g_rr<double>, G, kBlock, a_ga));
      b2 = b3;
    }
    CG_CUDA(h, add_kernel(body, &b3, b2, f_xp, G, kBlock, a_ga));
    prev = n;
  } else {
    CG_CUDA(h, cudaGraphCreate(&h->graph_it, 0));
    cudaGraphNode_t pi = nullptr, ci;
    for (int u = 0; u < unroll; ++u) {
      CG_CUDA(h, add_kernel(h->graph_it, &ci, pi, f_spmv, Gq, kBlock, a_ga));
      pi = ci;
      CG_CUDA(h, add_kernel(h->graph_it, &ci, pi, f_r, G, kBlock, a_ga));
      pi = ci;
      if (with_rr) {
        CG_CUDA(h, add_kernel(h->graph_it, &ci, pi, (const void*)g_rr<double>, G, kBlock, a_ga));
        pi = ci;
      }
      CG_CUDA(h, add_kernel(h->graph_it, &ci, pi, f_xp, G, kBlock, a_ga));
      pi = ci;
    }
    CG_CUDA(h, cudaGraphInstantiate(&h->gexec_it, h->graph_it, 0));
    CG_CUDA(h, cudaGraphCreate(&h->graph_ep, 0));
    ep = h->graph_ep;
    prev = nullptr;
  }
  // epilogue: flush on breakdown, true residual, final status
  CG_CUDA(h, add_kernel(ep, &n, prev, f_flush, G, kBlock, a_ga));
  prev = n;
  CG_CUDA(h, add_kernel(ep, &n, prev, (const void*)spmv_kernel<double>, Gs, kBlock, a_spmv));
  prev = n;
  CG_CUDA(h, add_kernel(ep, &n, prev, (const void*)g_true, G, kBlock, a_ga));
  prev = n;
  CG_CUDA(h, add_kernel(ep, &n, prev, (const void*)g_final64, 1, 32, a_ga));
  CG_CUDA(h, cudaGraphInstantiate(&h->gexec, g, 0));
  if (unroll > 0) CG_CUDA(h, cudaGraphInstantiate(&h->gexec_ep, h->graph_ep, 0));
  h->gkey_unroll = unroll;
  h->gkey_b = P.b;
  h->gkey_x = P.x;
  h->gkey_tol = P.tol;
  h->gkey_maxit = P.maxit;
  h->gkey_jac = jac;
  return CG_OK;
}

constexpr int64_t kGraphMinRows = 1 << 18;  // auto mode: graph loop from this many rows (fp64)
constexpr int64_t kClusterAutoRows = 16384;  // auto mode: the cluster form up to this many rows (fp64)
constexpr int kUnrollIters = 8;               // iterations per launch of the unrolled form

// fp64 solve through the graph form of the loop; restarts (true residual
// missing tol after the recursive test passed) relaunch the graph from x.
cg_status solve_graph64(cg_handle* h, const SolveParams& P, bool jac, int unroll,
                        int32_t* iters_out, double* relres_out) {
  if (!h->gexec || h->gkey_b != P.b || h->gkey_x != P.x || h->gkey_tol != P.tol ||
      h->gkey_maxit != P.maxit || h->gkey_jac != (int)jac || h->gkey_unroll != unroll) {
    cg_status s = build_graph64(h, P, jac, unroll);
    if (s != CG_OK) return s;
  }
  CG_CUDA(h, cudaMemsetAsync(h->gs, 0, sizeof(GState), h->stream));
  CG_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  int restarts = 0, status;
  int64_t launches = 0;
  int k_prev = 0;
  for (;;) {
    CG_CUDA(h, cudaGraphLaunch(h->gexec, h->stream));
    launches += 7;  // prologue 3 + epilogue 4
    if (unroll > 0) {
      for (;;) {  // iteration graphs until the loop state leaves kRunning
        CG_CUDA(h, cudaMemcpyAsync(h->host_gs, h->gs, sizeof(GState), cudaMemcpyDeviceToHost, h->stream));
        CG_CUDA(h, cudaStreamSynchronize(h->stream));
        if (h->host_gs->status != kRunning) break;
        CG_CUDA(h, cudaGraphLaunch(h->gexec_it, h->stream));
        launches += (jac && h->dmin != h->dmax ? 4 : 3) * unroll;
      }
      CG_CUDA(h, cudaGraphLaunch(h->gexec_ep, h->stream));
    }
    CG_CUDA(h, cudaMemcpyAsync(h->host_gs, h->gs, sizeof(GState), cudaMemcpyDeviceToHost, h->stream));
    CG_CUDA(h, cudaStreamSynchronize(h->stream));
    status = h->host_gs->status;
    if (unroll == 0) launches += (jac && h->dmin != h->dmax ? 4 : 3) * (int64_t)(h->host_gs->k - k_prev);
    k_prev = h->host_gs->k;
    if (status != kNeedRestart) break;
    if (h->host_gs->k >= P.maxit || restarts >= P.max_restarts) {
      status = kNotConverged;
      break;
    }
    ++restarts;
  }
  CG_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  CG_CUDA(h, cudaEventSynchronize(h->ev1));
  float ms = 0.0f;
  CG_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  const GState& gs = *h->host_gs;
  h->last.status = status;
  h->last.iters = gs.k;
  h->last.restarts = restarts;
  h->last.grid_ctas = h->grid_graph;
  h->last.relres_true = gs.relres_true;
  h->last.relres_rec = gs.bb > 0.0 ? sqrt(gs.rr) / sqrt(gs.bb) : 0.0;
  h->last.kernel_ms = ms;
  h->last.loop_form = unroll > 0 ? 3 : 2;
  h->last.kernel_launches = (int32_t)std::min<int64_t>(launches, INT32_MAX);
  const int64_t n = h->n, nnz = h->nnz;
  h->last.bytes_moved = (12 * nnz + 4 * (n + 1) + (jac ? 104 : 88) * n) * (int64_t)gs.k;
  const int64_t ent = h->sell_entries + h->nnz_long;
  h->last.kernel_bytes_per_iter = (h->dia ? 8 : 12) * ent + 4 * (int64_t)h->nlong + 80 * n +
                                  (jac && h->dmin != h->dmax ? 8 : 0) * n + loop_index_bytes(h);
  if (iters_out) *iters_out = gs.k;
  if (relres_out) *relres_out = gs.relres_true;
  if (status < 0) return fail(h, (cg_status)status, std::string("cg_solve: ") + cg_status_string(status));
  return (cg_status)status;
}

// Build the graph form of an fp32-inner / fp64-outer refinement solve.
cg_status build_graph_ir(cg_handle* h, const SolveParams& P, bool jac) {
  destroy_graph(&h->gexec, &h->graph);
  destroy_graph(&h->gexec_it, &h->graph_it);
  destroy_graph(&h->gexec_ep, &h->graph_ep);
  cudaGraph_t g;
  CG_CUDA(h, cudaGraphCreate(&g, 0));
  h->graph = g;
  cudaGraphConditionalHandle outer_h, inner_h;
  CG_CUDA(h, cudaGraphConditionalHandleCreate(&outer_h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams op{};
  op.type = cudaGraphNodeTypeConditional;
  op.conditional.handle = outer_h;
  op.conditional.type = cudaGraphCondTypeWhile;
  op.conditional.size = 1;
  cudaGraphNode_t on;
  CG_CUDA(h, cudaGraphAddNode(&on, g, nullptr, nullptr, 0, &op));
  cudaGraph_t ob = op.conditional.phGraph_out[0];
  CG_CUDA(h, cudaGraphConditionalHandleCreate(&inner_h, ob, 0, cudaGraphCondAssignDefault));
  const void* f_spmv = spmv_kernel_for<float>(h->uniform_w, h->dia != 0, jac, h->csr != 0);
  const unsigned G = (unsigned)h->grid_graph;
  const unsigned Gq = (unsigned)std::max(1, std::min(max_coresident(f_spmv, h->sm_count), h->grid_part));
  GArgs ga{P, h->gs, inner_h, outer_h, Gq, G};
  Csr<double> A = P.A;
  const double* x = P.x;
  double* q = P.V64.q;
  const unsigned Gs = spmv_grid(h);
  void* a_spmv[] = {&A, &x, &q};
  void* a_ga[] = {&ga};
  const bool with_rr = jac && h->dmin != h->dmax;
  cudaGraphNode_t n, prev;
  CG_CUDA(h, add_kernel(ob, &n, nullptr, (const void*)spmv_kernel<double>, Gs, kBlock, a_spmv));
  prev = n;
  CG_CUDA(h, add_kernel(ob, &n, prev, jac ? (const void*)g_res_ir<true> : (const void*)g_res_ir<false>,
                        G, kBlock, a_ga));
  prev = n;
  CG_CUDA(h, add_kernel(ob, &n, prev, (const void*)g_start_ir<true>, 1, 32, a_ga));
  prev = n;
  cudaGraphNodeParams ip{};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = inner_h;
  ip.conditional.type = cudaGraphCondTypeWhile;
  ip.conditional.size = 1;
  CG_CUDA(h, cudaGraphAddNode(&n, ob, &prev, nullptr, 1, &ip));
  cudaGraph_t ib = ip.conditional.phGraph_out[0];
  cudaGraphNode_t b1, b2, b3;
  CG_CUDA(h, add_kernel(ib, &b1, nullptr, f_spmv, Gq, kBlock, a_ga));
  CG_CUDA(h, add_kernel(ib, &b2, b1, jac ? (const void*)g_upd_r<float, true> : (const void*)g_upd_r<float, false>,
                        G, kBlock, a_ga));
  if (with_rr) {
    CG_CUDA(h, add_kernel(ib, &b3, b2, (const void*)g_rr<float>, G, kBlock, a_ga));
    b2 = b3;
  }
  CG_CUDA(h, add_kernel(ib, &b3, b2,
                        jac ? (const void*)g_upd_xp<float, true, true, true>
                            : (const void*)g_upd_xp<float, false, true, true>,
                        G, kBlock, a_ga));
  CG_CUDA(h, add_kernel(g, &n, on, (const void*)g_flush_ir, G, kBlock, a_ga));
  CG_CUDA(h, cudaGraphInstantiate(&h->gexec, g, 0));
  h->gkey_unroll = -2;  // marks the refinement graph
  h->gkey_b = P.b;
  h->gkey_x = P.x;
  h->gkey_tol = P.tol;
  h->gkey_maxit = P.maxit;
  h->gkey_jac = jac;
  h->gkey_tol_in = P.tol_in;
  h->gkey_outer = P.max_restarts;
  return CG_OK;
}

cg_status solve_graph_ir(cg_handle* h, const SolveParams& P, bool jac, int32_t* iters_out,
                         double* relres_out) {
  if (!h->gexec || h->gkey_unroll != -2 || h->gkey_b != P.b || h->gkey_x != P.x ||
      h->gkey_tol != P.tol || h->gkey_maxit != P.maxit || h->gkey_jac != (int)jac ||
      h->gkey_tol_in != P.tol_in || h->gkey_outer != P.max_restarts) {
    cg_status s = build_graph_ir(h, P, jac);
    if (s != CG_OK) return s;
  }
  CG_CUDA(h, cudaMemsetAsync(h->gs, 0, sizeof(GState), h->stream));
  CG_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  CG_CUDA(h, cudaGraphLaunch(h->gexec, h->stream));
  CG_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  CG_CUDA(h, cudaMemcpyAsync(h->host_gs, h->gs, sizeof(GState), cudaMemcpyDeviceToHost, h->stream));
  CG_CUDA(h, cudaStreamSynchronize(h->stream));
  float ms = 0.0f;
  CG_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  const GState& gs = *h->host_gs;
  const int status = gs.status;
  const int64_t n = h->n, nnz = h->nnz;
  h->last.status = status;
  h->last.iters = gs.k;
  h->last.restarts = gs.outer;
  h->last.grid_ctas = h->grid_graph;
  h->last.relres_true = gs.relres_true;
  h->last.relres_rec = gs.relres_true;
  h->last.kernel_ms = ms;
  h->last.loop_form = 2;
  const bool with_rr = jac && h->dmin != h->dmax;
  h->last.kernel_launches = (int32_t)std::min<int64_t>(
      3 * (int64_t)(gs.outer + 1) + (with_rr ? 4 : 3) * (int64_t)gs.k + 1, INT32_MAX);
  h->last.bytes_moved = (8 * nnz + 4 * (n + 1) + (jac ? 52 : 44) * n) * (int64_t)gs.k;
  const int64_t ent = h->sell_entries + h->nnz_long;
  const int64_t cb = h->dia ? 0 : 4;
  h->last.kernel_bytes_per_iter = (4 + cb) * ent + 4 * (int64_t)h->nlong + (with_rr ? 44 : 40) * n +
                                  loop_index_bytes(h);
  if (iters_out) *iters_out = gs.k;
  if (relres_out) *relres_out = gs.relres_true;
  if (status < 0) return fail(h, (cg_status)status, std::string("cg_solve: ") + cg_status_string(status));
  return (cg_status)status;
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
  h->host_rowptr.resize((size_t)n + 1);
  std::vector<int32_t>& hrp = h->host_rowptr;
  e = cudaMemcpy(hrp.data(), rowptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "cg_create: rowptr copy"));
  if (hrp[0] != 0) return bail(fail(h, CG_ERR_INVALID, "cg_create: rowptr[0] != 0"));
  for (int64_t i = 0; i < n; ++i)
    if (hrp[(size_t)i + 1] < hrp[(size_t)i])
      return bail(fail(h, CG_ERR_INVALID, "cg_create: rowptr decreases at row " + std::to_string(i)));
  h->nnz = hrp[(size_t)n];
  if (h->nnz > 0 && (!colind || !vals))
    return bail(fail(h, CG_ERR_INVALID, "cg_create: colind/vals NULL with nnz > 0"));

  std::vector<int32_t> rb = build_row_blocks(hrp.data(), n, &h->long_rows);
  h->nrb = (int32_t)(rb.size() - 1);
  const size_t nv = (size_t)std::max<int64_t>(n, 1);
  e = cudaMalloc(&h->rb, sizeof(int32_t) * rb.size());
  if (e == cudaSuccess) e = cudaMemcpy(h->rb, rb.data(), sizeof(int32_t) * rb.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->diag, sizeof(double) * nv);
  if (e == cudaSuccess) e = cudaMalloc(&h->ndiag, sizeof(int32_t) * nv);
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
    validate_kernel<<<grid_for(n), 256>>>(n, rowptr, colind, vals, h->diag, h->ndiag, cnt);
    e = cudaGetLastError();
  }
  unsigned long long hc[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost);
  if (cnt) cudaFree(cnt);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "cg_create: validation"));
  if (hc[0] != 0)
    return bail(fail(h, CG_ERR_INVALID, "cg_create: " + std::to_string(hc[0]) + " column indices outside [0, n)"));
  h->jacobi_ok = (hc[1] == 0);
  if (h->jacobi_ok && n > 0) {
    unsigned long long* mm = nullptr;
    unsigned long long hmm[2] = {~0ull, 0ull};
    e = cudaMalloc(&mm, sizeof(hmm));
    if (e == cudaSuccess) e = cudaMemcpy(mm, hmm, sizeof(hmm), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      diag_range_kernel<<<std::min<unsigned>(grid_for(n), 1024u), 256>>>(n, h->diag, mm);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(hmm, mm, sizeof(hmm), cudaMemcpyDeviceToHost);
    if (mm) cudaFree(mm);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cg_create: diagonal range"));
    std::memcpy(&h->dmin, &hmm[0], sizeof(double));
    std::memcpy(&h->dmax, &hmm[1], sizeof(double));
  }

  // persistent-kernel residency (the smallest over the kernels we may launch)
  const int g1 = max_coresident(pcg64_kernel<true>, h->sm_count);
  const int g2 = max_coresident(pcg64_kernel<false>, h->sm_count);
  const int g3 = std::min(max_coresident(pcg_ir_kernel<true, false>, h->sm_count),
                          max_coresident(pcg_ir_kernel<true, true>, h->sm_count));
  const int g4 = std::min(max_coresident(pcg_ir_kernel<false, false>, h->sm_count),
                          max_coresident(pcg_ir_kernel<false, true>, h->sm_count));
  h->grid_max = std::min(std::min(g1, g2), std::min(g3, g4));
  const int g5 = std::min(std::min(max_coresident(g_upd_r<double, true>, h->sm_count),
                                   max_coresident(g_upd_r<double, false>, h->sm_count)),
                          max_coresident(g_upd_xp<float, true, true, true>, h->sm_count));
  const int g6 = std::min(max_coresident(g_upd_xp<double, true, false, true>, h->sm_count),
                          max_coresident(g_res64<true>, h->sm_count));
  h->grid_graph = std::min(g5, g6);
  h->grid_part = 64 * h->sm_count;  // bounds every loop kernel's grid
  if (h->grid_max <= 0 || h->grid_graph <= 0 || h->grid_max > h->grid_part || h->grid_graph > h->grid_part)
    return bail(fail(h, CG_ERR_CUDA, "cg_create: occupancy query failed"));
  e = cudaMalloc(&h->part, sizeof(double) * (size_t)kParts * (size_t)h->grid_part);
  if (e == cudaSuccess) e = cudaMalloc(&h->gs, sizeof(GState));
  if (e == cudaSuccess) e = cudaMallocHost(&h->host_gs, sizeof(GState));
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
      h->tol_in_set = true;
      return CG_OK;
    case CG_OPT_IR_MAX_OUTER:
      if (!(value >= 0 && value <= 1000)) break;
      h->max_outer = (int)value;
      return CG_OK;
    case CG_OPT_DEBUG_SKIP_ARRIVAL:
      if (!(value >= 0 && value < 4e9)) break;
      h->skip_seq = (unsigned)value;
      return CG_OK;
    case CG_OPT_PHASE_TIMERS:
      if (!(value == 0 || value == 1)) break;
      h->timers = (int)value;
      return CG_OK;
    case CG_OPT_LOOP_MODE:
      if (!(value == 0 || value == 1 || value == 2 || value == 3 || value == 4)) break;
      h->loop_mode = (int)value;
      return CG_OK;
    default:
      break;
  }
  return fail(h, CG_ERR_INVALID, "cg_set_option: bad option or value");
}

cg_status cg_spmv(cg_handle* h, const double* x, double* y) {
  if (!h) return CG_ERR_INVALID;
  if (h->batch) return fail(h, CG_ERR_INVALID, "cg_spmv: batch handle (use cg_solve_batch)");
  if (h->n == 0) return CG_OK;
  if (!x || !y || x == y) return fail(h, CG_ERR_INVALID, "cg_spmv: x/y NULL or aliased");
  const Csr<double> A = make_csr(h);
  spmv_kernel<double><<<spmv_grid(h), kBlock, 0, h->stream>>>(A, x, y);
  CG_CUDA(h, cudaGetLastError());
  return CG_OK;
}

}  // extern "C"

namespace {

// Loop matrix (scaled with Jacobi, unscaled otherwise) and work vectors for
// one precision, built once per handle.
cg_status prepare_impl(cg_handle* h, bool jac, bool fp64) {
  cg_status s = ensure_offdiag(h);
  if (s == CG_OK) s = ensure_vectors<double>(h, &h->r, &h->p, &h->q, &h->xh);
  if (s == CG_OK && fp64) s = ensure_vals<double>(h, &h->sval64[jac], &h->lval64[jac], jac);
  if (s == CG_OK && !fp64) s = ensure_vals<float>(h, &h->sval32[jac], &h->lval32[jac], jac);
  if (s == CG_OK && !fp64) s = ensure_vectors<float>(h, &h->r32, &h->p32, &h->q32, &h->xh32);
  return s;
}

SolveParams make_solve_params(const cg_handle* h, bool jac, const double* b, double* x, double tol,
                              int32_t maxit, bool fp64, bool carry) {
  SolveParams P{};
  P.A = make_csr(h);
  P.S64 = make_sell<double>(h, h->sval64[jac], h->lval64[jac], h->diag, h->disq);
  P.S32 = make_sell<float>(h, h->sval32[jac], h->lval32[jac], h->diag32, h->disq32);
  P.V64 = LoopVecs<double>{h->r, h->p, h->q, h->xh};
  P.V32 = LoopVecs<float>{h->r32, h->p32, h->q32, h->xh32};
  P.b = b;
  P.x = x;
  P.dsq = h->dsq;
  P.disq = h->disq;
  P.part = h->part;
  P.pstride = h->grid_part;
  P.st = h->st;
  P.tol = tol;
  P.tol_in = h->tol_in_set ? h->tol_in : (carry ? kRuTolInner : kIrTolInner);
  P.maxit = maxit;
  P.max_restarts = fp64 ? h->max_restarts : h->max_outer;
  P.timeout_ns = (uint64_t)(h->timeout_ms * 1e6);
  P.skip_seq = h->skip_seq;
  P.timers = h->timers;
  return P;
}

cg_status check_precond_precision(cg_handle* h, int32_t precond, int32_t precision, const char* who) {
  if (precond != CG_PRECOND_NONE && precond != CG_PRECOND_JACOBI && precond != CG_PRECOND_FSAI)
    return fail(h, CG_ERR_INVALID, std::string(who) + ": unknown preconditioner");
  if (precision != CG_PREC_FP64 && precision != CG_PREC_FP32_IR && precision != CG_PREC_FP32_RU)
    return fail(h, CG_ERR_INVALID, std::string(who) + ": unknown precision");
  if (precond == CG_PRECOND_JACOBI && !h->jacobi_ok)
    return fail(h, CG_ERR_INVALID, std::string(who) + ": Jacobi needs a positive diagonal in every row");
  return CG_OK;
}

// Loop state for stand-alone launches of the loop SpMV: iterating, rho = 1,
// arrival counter clear (the kernel's last CTA forms alpha into this state).
__global__ void loop_spmv_state_kernel(GState* gs) {
  gs->status = kRunning;
  gs->rho = 1.0;
  gs->stop_abs = 0.0;
  gs->ctr_q = 0u;
}

// cg_solve after the preconditioner choice (FSAI only when the handle has a factor).
cg_status solve_impl(cg_handle* h, const double* b, double* x, double tol, int32_t maxit, int32_t precond,
                     int32_t precision, int32_t* iters_out, double* relres_out) {
  h->last = cg_solve_info{};
  if (!(tol >= 0.0) || maxit < 0) return fail(h, CG_ERR_INVALID, "cg_solve: tol < 0 or maxit < 0");
  const cg_status c = check_precond_precision(h, precond, precision, "cg_solve");
  if (c != CG_OK) return c;
  if (h->n == 0) {
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return CG_OK;
  }
  if (!b || !x) return fail(h, CG_ERR_INVALID, "cg_solve: b or x is NULL");
  if (!aligned16(b) || !aligned16(x)) return fail(h, CG_ERR_INVALID, "cg_solve: b and x must be 16-byte aligned");
  if (b == x) return fail(h, CG_ERR_INVALID, "cg_solve: b and x alias");
  const bool fsai = precond == CG_PRECOND_FSAI;
  const bool jac = precond == CG_PRECOND_JACOBI;  // FSAI runs on the unscaled matrix
  const bool fp64 = precision == CG_PREC_FP64;
  const bool carry = precision == CG_PREC_FP32_RU;  // reliable updates: persistent form only
  // small fp64 systems: the whole loop inside one thread-block cluster (no loop matrix needed)
  if (!fsai && fp64 &&
      (h->loop_mode == 4 ||
       (h->loop_mode == 0 && h->grid_opt == 0 && h->skip_seq == 0 && h->timers == 0 &&
        h->n <= kClusterAutoRows && h->n <= cgi::cluster_max_rows())))
    return cgi::cluster_solve(h, b, x, tol, maxit, jac, iters_out, relres_out);
  cg_status s = prepare_impl(h, jac, fp64);
  if (s != CG_OK) return s;

  const int G = auto_grid(h);
  SolveParams P = make_solve_params(h, jac, b, x, tol, maxit, fp64, carry);
  if (fsai) return cgi::fsai_solve(h, P, fp64, carry, G, iters_out, relres_out);
  // auto: fp64 takes the graph form from kGraphMinRows rows; the refinement's
  // fp32 vector passes are short, so it stays in the persistent form
  const bool graph_mode = !carry && (h->loop_mode >= 2 || (h->loop_mode == 0 && fp64 && h->n >= kGraphMinRows));
  if (graph_mode && fp64)
    return solve_graph64(h, P, jac, h->loop_mode == 3 ? kUnrollIters : 0, iters_out, relres_out);
  if (graph_mode) return solve_graph_ir(h, P, jac, iters_out, relres_out);
  void* args[] = {&P};
  const void* fn;
  if (fp64)
    fn = jac ? (const void*)pcg64_kernel<true> : (const void*)pcg64_kernel<false>;
  else
    fn = carry ? (jac ? (const void*)pcg_ir_kernel<true, true> : (const void*)pcg_ir_kernel<false, true>)
               : (jac ? (const void*)pcg_ir_kernel<true, false> : (const void*)pcg_ir_kernel<false, false>);
  CG_CUDA(h, cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream));
  CG_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  CG_CUDA(h, cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kBlock), args, 0, h->stream));
  CG_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  CG_CUDA(h, cudaMemcpyAsync(h->host_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CG_CUDA(h, cudaStreamSynchronize(h->stream));
  float ms = 0.0f;
  CG_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  const DevState& ds = *h->host_st;
  cg_status status = ds.abort ? CG_ERR_TIMEOUT : (cg_status)ds.status;
  h->last.status = status;
  h->last.iters = ds.iters;
  h->last.restarts = ds.restarts;
  h->last.grid_ctas = G;
  h->last.relres_true = ds.relres_true;
  h->last.relres_rec = ds.relres_rec;
  h->last.kernel_ms = ms;
  h->last.loop_form = 1;
  h->last.kernel_launches = 1;
  // modelled bytes of the CG loop (three phases of Alg. 1 on the caller's CSR)
  const int64_t n = h->n, nnz = h->nnz;
  const int64_t per_iter = fp64 ? 12 * nnz + 4 * (n + 1) + (jac ? 104 : 88) * n
                                : 8 * nnz + 4 * (n + 1) + (jac ? 52 : 44) * n;
  h->last.bytes_moved = per_iter * (int64_t)ds.iters;
  // bytes this kernel's loop must move per iteration: the SELL-32 slices
  // (padding included), the long-row CSR and the vector streams
  const int64_t ent = h->sell_entries + h->nnz_long;
  const int64_t cb = h->dia ? 0 : 4;  // column bytes per entry
  const int64_t vb = 80 + (jac && h->dmin != h->dmax ? 8 : 0);  // vector bytes per row (fp64)
  h->last.kernel_bytes_per_iter = fp64 ? (8 + cb) * ent + 4 * (int64_t)h->nlong + vb * n
                                       : (4 + cb) * ent + 4 * (int64_t)h->nlong + vb / 2 * n;
  h->last.kernel_bytes_per_iter += loop_index_bytes(h);
  for (int j = 0; j < 6; ++j) h->last.phase_ms[j] = ds.tphase[j] * 1e-6;
  if (iters_out) *iters_out = ds.iters;
  if (relres_out) *relres_out = ds.relres_true;
  if (status == CG_ERR_TIMEOUT)
    return fail(h, status, "cg_solve: a bounded wait gave up (barrier " + std::to_string(ds.err_barrier) +
                               ", CTA " + std::to_string(ds.err_cta) + "); timed out");
  if (status < 0) return fail(h, status, std::string("cg_solve: ") + cg_status_string(status));
  return status;
}

}  // namespace

extern "C" {

cg_status cg_solve(cg_handle* h, const double* b, double* x, double tol, int32_t maxit,
                   int32_t precond, int32_t precision, int32_t* iters_out, double* relres_out) {
  if (!h) return CG_ERR_INVALID;
  if (h->batch) return fail(h, CG_ERR_INVALID, "cg_solve: batch handle (use cg_solve_batch)");
  int32_t used = precond;
  if (precond == CG_PRECOND_FSAI && !(h->fsai && h->fsai->kind)) used = CG_PRECOND_JACOBI;  // fallback
  const cg_status s = solve_impl(h, b, x, tol, maxit, used, precision, iters_out, relres_out);
  h->last.precond_used = used;
  return s;
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

cg_status cg_prepare(cg_handle* h, int32_t precond, int32_t precision) {
  if (!h) return CG_ERR_INVALID;
  if (h->batch) return fail(h, CG_ERR_INVALID, "cg_prepare: batch handle");
  const cg_status c = check_precond_precision(h, precond, precision, "cg_prepare");
  if (c != CG_OK) return c;
  if (h->n == 0) return CG_OK;
  const bool fp64 = precision == CG_PREC_FP64;
  cg_status s = prepare_impl(h, precond == CG_PRECOND_JACOBI, fp64);
  // FSAI without a factor solves with Jacobi: build that variant too
  if (s == CG_OK && precond == CG_PRECOND_FSAI && !(h->fsai && h->fsai->kind) && h->jacobi_ok)
    s = prepare_impl(h, true, fp64);
  return s;
}

cg_status cg_loop_spmv(cg_handle* h, int32_t precond, int32_t precision, const void* p, void* q, int32_t reps,
                       int64_t* bytes_out) {
  if (!h) return CG_ERR_INVALID;
  if (h->batch) return fail(h, CG_ERR_INVALID, "cg_loop_spmv: batch handle");
  const cg_status c = check_precond_precision(h, precond, precision, "cg_loop_spmv");
  if (c != CG_OK) return c;
  if (reps < 1) return fail(h, CG_ERR_INVALID, "cg_loop_spmv: reps < 1");
  if (h->n == 0) {
    if (bytes_out) *bytes_out = 0;
    return CG_OK;
  }
  if (!p || !q || p == q) return fail(h, CG_ERR_INVALID, "cg_loop_spmv: p/q NULL or aliased");
  if (!aligned16(p) || !aligned16(q)) return fail(h, CG_ERR_INVALID, "cg_loop_spmv: p and q must be 16-byte aligned");
  const bool jac = precond == CG_PRECOND_JACOBI;
  const bool fp64 = precision == CG_PREC_FP64;
  cg_status s = prepare_impl(h, jac, fp64);
  if (s != CG_OK) return s;
  SolveParams P = make_solve_params(h, jac, nullptr, nullptr, 0.0, 0, fp64, false);
  if (fp64) {
    P.V64.p = static_cast<double*>(const_cast<void*>(p));
    P.V64.q = static_cast<double*>(q);
  } else {
    P.V32.p = static_cast<float*>(const_cast<void*>(p));
    P.V32.q = static_cast<float*>(q);
  }
  const void* f = fp64 ? spmv_kernel_for<double>(h->uniform_w, h->dia != 0, jac, h->csr != 0)
                       : spmv_kernel_for<float>(h->uniform_w, h->dia != 0, jac, h->csr != 0);
  const unsigned Gq = (unsigned)std::max(1, std::min(max_coresident(f, h->sm_count), h->grid_part));
  GArgs ga{P, h->gs, 0, 0, Gq, (unsigned)h->grid_graph};
  void* args[] = {&ga};
  loop_spmv_state_kernel<<<1, 1, 0, h->stream>>>(h->gs);
  CG_CUDA(h, cudaGetLastError());
  for (int r = 0; r < reps; ++r)
    CG_CUDA(h, cudaLaunchKernel(f, dim3(Gq), dim3(kBlock), args, 0, h->stream));
  if (bytes_out) {
    // the entries of the loop matrix (8 B fp64 / 4 B fp32, plus a 4 B column
    // without the diagonal layout), p read once, q written
    const int64_t ent = h->sell_entries + h->nnz_long;
    const int64_t vb = fp64 ? 8 : 4, cb = h->dia ? 0 : 4;
    *bytes_out = (vb + cb) * ent + 4 * (int64_t)h->nlong + 2 * vb * h->n +
                 (jac ? 0 : vb * h->n) +  // the stored diagonal without Jacobi
                 loop_index_bytes(h);
  }
  return CG_OK;
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
