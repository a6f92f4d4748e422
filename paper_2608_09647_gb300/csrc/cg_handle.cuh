// Host-side state behind the opaque cg_handle of include/libcg.h (shared by
// the translation units of the library).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/libcg.h"
#include "cg_kernels.cuh"

namespace cg {
struct GState;                    // graph-form loop state (cg_graph.cuh)
}

using cg::DevState;
using cg::GState;
using cg::kMaxDiag;

struct BatchData;                 // batched solves (cg_batch.cu)
struct FsaiData;                  // FSAI preconditioner (cg_fsai.cu, cg_mlp.cu)

namespace cgi {
void batch_free(BatchData* b);
void fsai_free(FsaiData* f);
void set_create_error(const std::string& msg);  // message of cg_last_error(NULL)
cg_status ensure_offsets(cg_handle* h);         // cg_handle::offs_all, once (cg_api.cu)
// the loop in one thread-block cluster (cg_cluster.cu): fp64 CG / Jacobi-PCG of small systems
int64_t cluster_max_rows();
cg_status cluster_solve(cg_handle* h, const double* b, double* x, double tol, int32_t maxit, bool jac,
                        int32_t* iters_out, double* relres_out);
}  // namespace cgi

// Device memory owned by a handle.  The internal off-diagonal matrices and
// work vectors are built on first use of a precision / preconditioner.
struct cg_handle {
  int64_t n = 0, nnz = 0;
  const int32_t* rowptr = nullptr;  // borrowed caller CSR
  const int32_t* colind = nullptr;
  const double* vals = nullptr;
  int32_t* rb = nullptr;            // row blocks of the caller CSR
  int32_t nrb = 0;
  int64_t long_rows = 0;
  std::vector<int32_t> host_rowptr;
  // diagonal data
  double* diag = nullptr;           // A_ii (sum of stored diagonal entries)
  int32_t* ndiag = nullptr;         // diagonal entries per row
  double *dsq = nullptr, *disq = nullptr;
  float *diag32 = nullptr, *disq32 = nullptr;
  bool jacobi_ok = false;
  // off-diagonal loop matrix in SELL-32 form (+ compact CSR of long rows)
  int32_t nslices = 0;
  int32_t uniform_w = -1;           // every slice padded to this width (-1: variable)
  int32_t dia = 0;                  // sliced-diagonal layout (no column array)
  double dmin = 1.0, dmax = 1.0;    // range of A_ii (Jacobi)
  int32_t delta[kMaxDiag] = {};     // its diagonal offsets, ascending
  // every distinct off-diagonal offset j - i of the CSR, ascending (loop
  // layout, features of the learned factor); noffs_all = -1 when there are
  // more than kOffsAll, kOffsUnknown before cgi::ensure_offsets
  static constexpr int kOffsAll = 64;
  static constexpr int32_t kOffsUnknown = -2;
  int32_t noffs_all = kOffsUnknown;
  int32_t offs_all[kOffsAll] = {};
  int32_t* delta_dev = nullptr;
  int32_t* soff = nullptr;
  uint32_t* lmask = nullptr;
  int32_t csr = 0;                  // 1: the loop matrix is an off-diagonal CSR in row blocks
  int32_t *lrp = nullptr, *lrb = nullptr;  // its row pointers and row blocks
  int32_t lnrb = 0;
  int32_t* sperm = nullptr;         // SELL-C-sigma: row of each slice position (n = none)
  int32_t* spos = nullptr;          // and slice position of each row
  int32_t* scol = nullptr;
  int64_t sell_entries = 0;         // padded entries (multiple of 32)
  int64_t nnz_od = 0;
  int32_t nlong = 0;
  int32_t *lrow = nullptr, *lptr = nullptr, *lcol = nullptr;
  int64_t nnz_long = 0;
  double* sval64[2] = {nullptr, nullptr};  // [precond]: unscaled / Jacobi-scaled
  float* sval32[2] = {nullptr, nullptr};
  double* lval64[2] = {nullptr, nullptr};
  float* lval32[2] = {nullptr, nullptr};
  bool scol_written = false;
  // work vectors
  double *r = nullptr, *p = nullptr, *q = nullptr, *xh = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *xh32 = nullptr;
  double* part = nullptr;
  DevState* st = nullptr;
  DevState* host_st = nullptr;      // pinned
  double *stage_b = nullptr, *stage_x = nullptr;  // device staging of cg_solve_host (lazy)
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int sm_count = 0;
  int grid_max = 0;                 // co-resident CTAs of the persistent kernels
  int grid_opt = 0;                 // CG_OPT_GRID_CTAS (0 = auto)
  int max_restarts = 3;
  double timeout_ms = 2000.0;
  double tol_in = 1e-4;
  bool tol_in_set = false;          // CG_OPT_IR_TOL_INNER given (else the precision's default)
  int max_outer = 30;
  unsigned skip_seq = 0;
  int timers = 0;
  int loop_mode = 0;                // CG_OPT_LOOP_MODE (0 auto, 1 persistent, 2 graph)
  // graph form of the loop
  int grid_graph = 0;               // CTAs of the graph-mode vector kernels
  int grid_part = 0;                // partial-sum slots per kind (the largest grid of any loop kernel)
  GState* gs = nullptr;
  GState* host_gs = nullptr;        // pinned
  cudaGraph_t graph = nullptr, graph_it = nullptr, graph_ep = nullptr;
  cudaGraphExec_t gexec = nullptr, gexec_it = nullptr, gexec_ep = nullptr;
  int gkey_unroll = -1;
  const void* gkey_b = nullptr;     // the graph bakes in these solve arguments
  const void* gkey_x = nullptr;
  double gkey_tol = -1.0;
  int gkey_maxit = -1, gkey_jac = -1;
  double gkey_tol_in = -1.0;
  int gkey_outer = -1;
  cg_solve_info last{};
  std::string err;
  BatchData* batch = nullptr;       // set for handles made by cg_batch_create
  FsaiData* fsai = nullptr;         // FSAI factor (built on first use)
};

