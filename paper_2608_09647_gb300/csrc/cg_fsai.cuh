// FSAI preconditioner state of a handle (shared by cg_fsai.cu and cg_mlp.cu).
#pragma once

#include "cg_handle.cuh"

constexpr int kFsaiMaxRow = 16;   // longest row of tril(A) the factor supports
constexpr int kFsaiMaxCol = 32;   // longest column of tril(A) (row of G^T)
constexpr int kFsaiMaxDiag = 8;   // most offsets of tril(A) for the diagonal layout

struct FsaiData {
  int64_t ntril = 0;               // entries of tril(A) = nonzeros of G
  int32_t *trp = nullptr, *tci = nullptr;  // tril(A) pattern (CSR)
  int32_t* tsrc = nullptr;         // index of each tril entry in A's arrays
  double* g = nullptr;             // factor values in tril order
  int kind = 0;                    // 0 none, 1 classic, 2 learned, 3 set by the caller
  // ELL layouts for the loop: slot m of row i at [m n + i]
  int gw = 0, gtw = 0;
  int dia = 0, nd = 0;             // diagonal layout: its offset count and offsets
  int32_t doff[kFsaiMaxDiag] = {};
  int8_t* tslot = nullptr;         // diagonal slot of each tril entry
  int32_t *gsrc = nullptr, *gcol = nullptr;     // G
  double* gval64 = nullptr;
  float* gval32 = nullptr;
  int32_t *gtsrc = nullptr, *gtcol = nullptr;   // G^T
  double* gtval64 = nullptr;
  float* gtval32 = nullptr;
  // loop vectors beyond the handle's
  double *r0 = nullptr, *r1 = nullptr, *t = nullptr;
  float *r0_32 = nullptr, *r1_32 = nullptr, *t_32 = nullptr, *x_32 = nullptr;
  // learned factor: matrix offsets, work space
  int32_t* offs = nullptr;         // sorted distinct column offsets of A (device)
  int host_offs[9] = {};           // the same on the host
  int noffs = 0, ntslots = 0;      // their count; count of those <= 0
  int32_t* trow = nullptr;         // row of each tril entry
  double* work = nullptr;          // training work vectors
  double* rpart = nullptr;         // block partial sums of the loss kernels
  float* dout = nullptr;           // dLoss/do per tril entry
  float* gpart = nullptr;          // per-CTA partial parameter gradients
  float* mlp_o = nullptr;          // MLP output per tril entry
  float* a32 = nullptr;            // A's values in fp32 (feature inputs)
  float* d32 = nullptr;            // A_ii in fp32
  float* rs32 = nullptr;           // 1 / sqrt(A_ii) in fp32
  double* rs64 = nullptr;          // 1 / sqrt(A_ii) in fp64 (G from the outputs)
  float* params32 = nullptr;       // parameters given to cg_fsai_load (device, fp32)
  // graph forms of the fp32 refinement loop: one graph with nested WHILE
  // nodes, or (unrolled) an outer-step graph, an 8-iteration graph and an
  // epilogue graph relaunched by the host
  cudaGraph_t graph = nullptr, graph_it = nullptr, graph_ep = nullptr;
  cudaGraphExec_t gexec = nullptr, gexec_it = nullptr, gexec_ep = nullptr;
  const void* gkey_b = nullptr;
  const void* gkey_x = nullptr;
  double gkey_tol = -1.0, gkey_tol_in = -1.0;
  int gkey_maxit = -1, gkey_outer = -1, gkey_carry = -1, gkey_kind = -1, gkey_unroll = -1;
  int ggrid = 0;  // CTAs of the graph form's vector-phase kernels
};

namespace cgi {
cg_status fsai_pattern(cg_handle* h);
cg_status fsai_commit(cg_handle* h, int kind);
cg_status fsai_solve(cg_handle* h, const cg::SolveParams& P, bool fp64, bool carry, int grid,
                     int32_t* iters_out, double* relres_out);
}  // namespace cgi
