// Learned FSAI factor: a 32-64-64-1 MLP maps local features of every entry
// of tril(A) to that entry of G (inference), and its training loss (Kaporin
// number plus residual-history term) is differentiated back to the
// parameters (training).  Not in the paper.
//
// Precision: parameters and features in bf16, products accumulated in fp32
// on the tensor cores (mma.sync m16n8k16 bf16), h1 = bf16(relu(z1)), h2 =
// relu(z2) in fp32, output layer on the CUDA cores in fp32.  G, the loss and
// dLoss/dG in fp64.  Backward: dz2 and dz1 rounded to bf16 as tensor-core
// inputs (dh1 = dz2 W2, dW2 = dz2^T h1, dW1 = dz1^T x), bias gradients from
// the fp32 values; every sum over entries runs in a fixed order (per-CTA
// partials reduced in CTA order), so a gradient is reproducible bit for bit.
//
// Features of entry (i, j), d = diag(A), s(i,k) = A_ik / sqrt(d_i d_k):
//   [0:8] one-hot slot of j - i among the non-positive offsets of A,
//   [8] s(i,j), [9] log(d_j / d_i), [10:19] s(i, i + o_m), [19:28] s(j, j + o_m)
//   over the sorted distinct offsets o_m of A (at most 9), [28] 1, [29:32] 0.
// Output o: G_ij = o / sqrt(d_j) (j < i), G_ii = softplus(o + c0) / sqrt(d_i)
// with softplus(c0) = 1, so a zero output layer gives G = D^-1/2 (Jacobi).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cg_fsai.cuh"

using namespace cg;

namespace {

constexpr int kIn = CG_MLP_INPUTS, kHid = CG_MLP_HIDDEN, kNParams = CG_MLP_PARAMS;
constexpr int kOffW1 = 0, kOffB1 = kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid;
static_assert(kOffB3 + 1 == kNParams, "parameter layout");
constexpr int kMaxOffs = 9;
constexpr int kMlpThreads = 128;         // 4 warps x 16 entries per step
constexpr int kTileE = 64;               // entries per CTA step
constexpr int kW1S = kIn + 8;            // padded smem row strides (bf16 elements)
constexpr int kW2S = kHid + 8;
constexpr int kTS = kTileE + 8;          // transposed tiles: [feature][entry]

struct MlpArgs {
  int64_t n, ntril;
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ colind;
  const double* __restrict__ vals;
  const double* __restrict__ diag;
  const int32_t* __restrict__ trow;      // row of each tril entry
  const int32_t* __restrict__ tci;       // column of each tril entry
  const int32_t* __restrict__ tsrc;      // index of each tril entry in A's arrays
  const float* __restrict__ params;      // fp32 parameters (rounded to bf16 on load)
  const float* __restrict__ a32;         // A's values, A_ii and 1 / sqrt(A_ii) in fp32
  const float* __restrict__ d32;
  const float* __restrict__ rs32;
  int offs[kMaxOffs];
  int noffs, ntslots;
  double c0;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// d += a b for one 16x8x16 tile (bf16 inputs, fp32 accumulators).
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ int offset_slot(const MlpArgs& M, int off) {
  for (int m = 0; m < M.noffs; ++m)
    if (M.offs[m] == off) return m;
  return -1;
}

// Features of tril entry e into a 32-wide bf16 row: lanes 0-15 write the
// entry part and row i's entries, lanes 16-31 row j's entries and the tail.
__device__ void entry_features(const MlpArgs& M, int64_t e, bool upper_half, __nv_bfloat16* xr) {
  if (e >= M.ntril) {
    const int a = upper_half ? 16 : 0;
    for (int f = a; f < a + 16; ++f) xr[f] = __float2bfloat16_rn(0.0f);
    return;
  }
  // formed in fp32 from fp32 copies of A's values and diagonal (GB300 runs
  // fp64, conversions included, at 1/64 of the fp32 rate) and rounded to
  // bf16, the network's input precision
  const int i = M.trow[e], j = M.tci[e];
  const float si = M.rs32[i], sj = M.rs32[j];
  float f[19];
  if (!upper_half) {
    for (int k = 0; k < 19; ++k) f[k] = 0.0f;
    const int slot = offset_slot(M, j - i);  // always one of the first ntslots
    if (slot >= 0 && slot < 8) f[slot] = 1.0f;
    f[8] = M.a32[M.tsrc[e]] * si * sj;
    f[9] = logf(M.d32[j] / M.d32[i]);
    for (int k = M.rowptr[i]; k < M.rowptr[i + 1]; ++k) {
      const int c = M.colind[k];
      const int s = offset_slot(M, c - i);
      if (s >= 0) f[10 + s] = M.a32[k] * si * M.rs32[c];
    }
    for (int k = 0; k < 19; ++k) xr[k] = __float2bfloat16_rn(f[k]);
  } else {
    for (int k = 0; k < 9; ++k) f[k] = 0.0f;
    for (int k = M.rowptr[j]; k < M.rowptr[j + 1]; ++k) {
      const int c = M.colind[k];
      const int s = offset_slot(M, c - j);
      if (s >= 0) f[s] = M.a32[k] * sj * M.rs32[c];
    }
    for (int k = 0; k < 9; ++k) xr[19 + k] = __float2bfloat16_rn(f[k]);
    xr[28] = __float2bfloat16_rn(1.0f);
    for (int k = 29; k < 32; ++k) xr[k] = __float2bfloat16_rn(0.0f);
  }
}

// Shared parameters of a CTA: bf16 weights (W1, W2 and, for backward, W2^T)
// and fp32 biases / output layer.
struct __align__(16) SmemW {
  __nv_bfloat16 w1[kHid * kW1S];
  __nv_bfloat16 w2[kHid * kW2S];
  float b1[kHid], b2[kHid], w3[kHid];
  float b3;
};

__device__ void load_weights(const MlpArgs& M, SmemW& S, __nv_bfloat16* w2t) {
  for (int k = threadIdx.x; k < kHid * kIn; k += blockDim.x)
    S.w1[(k / kIn) * kW1S + k % kIn] = __float2bfloat16_rn(M.params[kOffW1 + k]);
  for (int k = threadIdx.x; k < kHid * kHid; k += blockDim.x) {
    const __nv_bfloat16 v = __float2bfloat16_rn(M.params[kOffW2 + k]);
    S.w2[(k / kHid) * kW2S + k % kHid] = v;
    if (w2t) w2t[(k % kHid) * kW2S + k / kHid] = v;
  }
  for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
    S.b1[k] = __bfloat162float(__float2bfloat16_rn(M.params[kOffB1 + k]));
    S.b2[k] = __bfloat162float(__float2bfloat16_rn(M.params[kOffB2 + k]));
    S.w3[k] = __bfloat162float(__float2bfloat16_rn(M.params[kOffW3 + k]));
  }
  if (threadIdx.x == 0) S.b3 = __bfloat162float(__float2bfloat16_rn(M.params[kOffB3]));
}

// The forward pass of a warp's 16 entries (features already in xs, 16 rows
// of kW1S): z1 (C fragments, 8 n-tiles), h1 (A fragments, 4 k-steps), z2, and
// o for rows g and g + 8 (every lane of the group holds them).
struct Fwd {
  float z1[8][4];
  uint32_t h1[4][4];
  float z2[8][4];
  float o[2];
};

__device__ __forceinline__ void forward16(const SmemW& S, const __nv_bfloat16* xs, Fwd& F) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t xa[2][4];
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    xa[kk][0] = lds32(xs + g * kW1S + 16 * kk + 2 * t);
    xa[kk][1] = lds32(xs + (g + 8) * kW1S + 16 * kk + 2 * t);
    xa[kk][2] = lds32(xs + g * kW1S + 16 * kk + 8 + 2 * t);
    xa[kk][3] = lds32(xs + (g + 8) * kW1S + 16 * kk + 8 + 2 * t);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float bl = S.b1[8 * j + 2 * t], bh = S.b1[8 * j + 2 * t + 1];
    F.z1[j][0] = bl;
    F.z1[j][1] = bh;
    F.z1[j][2] = bl;
    F.z1[j][3] = bh;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const __nv_bfloat16* wr = S.w1 + (8 * j + g) * kW1S + 16 * kk + 2 * t;
      mma16816(F.z1[j], xa[kk], lds32(wr), lds32(wr + 8));
    }
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const float* lo = F.z1[2 * kk];
    const float* hi = F.z1[2 * kk + 1];
    F.h1[kk][0] = pack_bf16(fmaxf(lo[0], 0.0f), fmaxf(lo[1], 0.0f));
    F.h1[kk][1] = pack_bf16(fmaxf(lo[2], 0.0f), fmaxf(lo[3], 0.0f));
    F.h1[kk][2] = pack_bf16(fmaxf(hi[0], 0.0f), fmaxf(hi[1], 0.0f));
    F.h1[kk][3] = pack_bf16(fmaxf(hi[2], 0.0f), fmaxf(hi[3], 0.0f));
  }
  float og = 0.0f, og8 = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float bl = S.b2[8 * j + 2 * t], bh = S.b2[8 * j + 2 * t + 1];
    F.z2[j][0] = bl;
    F.z2[j][1] = bh;
    F.z2[j][2] = bl;
    F.z2[j][3] = bh;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const __nv_bfloat16* wr = S.w2 + (8 * j + g) * kW2S + 16 * kk + 2 * t;
      mma16816(F.z2[j], F.h1[kk], lds32(wr), lds32(wr + 8));
    }
    const float wl = S.w3[8 * j + 2 * t], wh = S.w3[8 * j + 2 * t + 1];
    og = fmaf(wl, fmaxf(F.z2[j][0], 0.0f), og);
    og = fmaf(wh, fmaxf(F.z2[j][1], 0.0f), og);
    og8 = fmaf(wl, fmaxf(F.z2[j][2], 0.0f), og8);
    og8 = fmaf(wh, fmaxf(F.z2[j][3], 0.0f), og8);
  }
  og += __shfl_xor_sync(0xffffffffu, og, 1);
  og += __shfl_xor_sync(0xffffffffu, og, 2);
  og8 += __shfl_xor_sync(0xffffffffu, og8, 1);
  og8 += __shfl_xor_sync(0xffffffffu, og8, 2);
  F.o[0] = og + S.b3;
  F.o[1] = og8 + S.b3;
}

__device__ __forceinline__ double softplus_d(double x) {
  return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
}
__device__ __forceinline__ double sigmoid_d(double x) {
  return x >= 0.0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x));
}

// Inference / training forward: the output o of every tril entry (G from o in
// g_diag_kernel / g_offdiag_kernel).
__global__ void __launch_bounds__(kMlpThreads) mlp_forward_kernel(MlpArgs M, float* __restrict__ o_out) {
  __shared__ __align__(16) SmemW S;
  __shared__ __align__(16) __nv_bfloat16 xs[4][16 * kW1S];  // 32-bit fragment loads need 4-byte alignment
  load_weights(M, S, nullptr);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  for (int64_t base = (int64_t)blockIdx.x * kTileE; base < M.ntril; base += (int64_t)gridDim.x * kTileE) {
    const int64_t wb = base + 16 * warp;
    entry_features(M, wb + (lane & 15), lane >= 16, xs[warp] + (lane & 15) * kW1S);
    __syncwarp();
    Fwd F;
    forward16(S, xs[warp], F);
    if (t == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t e = wb + g + 8 * h;
        if (e < M.ntril) o_out[e] = F.o[h];
      }
    }
    __syncwarp();
  }
}

// Backward: per CTA, partial gradients of every parameter over its tiles
// (written to part[blockIdx.x * kNParams + k]).
struct __align__(16) SmemB {
  SmemW w;
  __nv_bfloat16 w2t[kHid * kW2S];
  __nv_bfloat16 xs[4][16 * kW1S];
  __nv_bfloat16 dz2t[kHid * kTS];   // [unit][entry]
  __nv_bfloat16 h1t[kHid * kTS];
  __nv_bfloat16 dz1t[kHid * kTS];
  __nv_bfloat16 xt[kIn * kTS];
  float red[4][3 * kHid];           // per-warp column sums: db1, db2, dW3
  float red3[4];
};

__global__ void __launch_bounds__(kMlpThreads) mlp_backward_kernel(MlpArgs M, const float* __restrict__ dout,
                                                                     float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemB& S = *reinterpret_cast<SmemB*>(smem_raw);
  load_weights(M, S.w, S.w2t);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  float dw2[8][4], dw1[4][4];
  float db1[16], db2[16], dw3[16], db3 = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) dw2[j][c] = 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) dw1[j][c] = 0.0f;
#pragma unroll
  for (int c = 0; c < 16; ++c) db1[c] = db2[c] = dw3[c] = 0.0f;

  for (int64_t base = (int64_t)blockIdx.x * kTileE; base < M.ntril; base += (int64_t)gridDim.x * kTileE) {
    const int64_t wb = base + 16 * warp;
    __nv_bfloat16* xs = S.xs[warp];
    entry_features(M, wb + (lane & 15), lane >= 16, xs + (lane & 15) * kW1S);
    __syncwarp();
    Fwd F;
    forward16(S.w, xs, F);
    float dg = 0.0f, dg8 = 0.0f;  // dLoss/do of rows g, g + 8 (0 past the end)
    if (wb + g < M.ntril) dg = dout[wb + g];
    if (wb + g + 8 < M.ntril) dg8 = dout[wb + g + 8];
    if (t == 0) db3 += dg + dg8;
    // dz2 = dout w3 [z2 > 0]; dW3 += dout h2; db2 += dz2
    float dz2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = 8 * j + 2 * t + (c & 1);
        const float dd = c < 2 ? dg : dg8;
        const float z = F.z2[j][c];
        dw3[2 * j + (c & 1)] = fmaf(dd, fmaxf(z, 0.0f), dw3[2 * j + (c & 1)]);
        const float v = z > 0.0f ? dd * S.w.w3[col] : 0.0f;
        dz2[j][c] = v;
        db2[2 * j + (c & 1)] += v;
      }
    }
    // dz2 as bf16 A fragments; dh1 = dz2 W2 (B = W2^T rows), dz1 = dh1 [z1 > 0]
    uint32_t dza[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      dza[kk][0] = pack_bf16(dz2[2 * kk][0], dz2[2 * kk][1]);
      dza[kk][1] = pack_bf16(dz2[2 * kk][2], dz2[2 * kk][3]);
      dza[kk][2] = pack_bf16(dz2[2 * kk + 1][0], dz2[2 * kk + 1][1]);
      dza[kk][3] = pack_bf16(dz2[2 * kk + 1][2], dz2[2 * kk + 1][3]);
    }
    float dz1[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const __nv_bfloat16* wr = S.w2t + (8 * j + g) * kW2S + 16 * kk + 2 * t;
        mma16816(acc, dza[kk], lds32(wr), lds32(wr + 8));
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float v = F.z1[j][c] > 0.0f ? acc[c] : 0.0f;
        dz1[j][c] = v;
        db1[2 * j + (c & 1)] += v;
      }
    }
    // transposed bf16 tiles for the weight gradients: [unit][entry]
    const int er = 16 * warp + g;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = 8 * j + 2 * t + (c & 1);
        const int ent = er + (c < 2 ? 0 : 8);
        S.dz2t[col * kTS + ent] = __float2bfloat16_rn(dz2[j][c]);
        S.dz1t[col * kTS + ent] = __float2bfloat16_rn(dz1[j][c]);
        S.h1t[col * kTS + ent] = __float2bfloat16_rn(fmaxf(F.z1[j][c], 0.0f));
      }
    }
    for (int k = lane; k < 16 * kIn; k += 32) {
      const int r = k / kIn, f = k % kIn;
      S.xt[f * kTS + 16 * warp + r] = xs[r * kW1S + f];
    }
    __syncthreads();
    // warp w: rows [16w, 16w + 16) of dW2 (K = the tile's 64 entries) and of dW1
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t a2[4], a1[4];
      const __nv_bfloat16* p2 = S.dz2t + (16 * warp + g) * kTS + 16 * kk + 2 * t;
      a2[0] = lds32(p2);
      a2[1] = lds32(p2 + 8 * kTS);
      a2[2] = lds32(p2 + 8);
      a2[3] = lds32(p2 + 8 * kTS + 8);
      const __nv_bfloat16* p1 = S.dz1t + (16 * warp + g) * kTS + 16 * kk + 2 * t;
      a1[0] = lds32(p1);
      a1[1] = lds32(p1 + 8 * kTS);
      a1[2] = lds32(p1 + 8);
      a1[3] = lds32(p1 + 8 * kTS + 8);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const __nv_bfloat16* hb = S.h1t + (8 * j + g) * kTS + 16 * kk + 2 * t;
        mma16816(dw2[j], a2, lds32(hb), lds32(hb + 8));
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat16* xb = S.xt + (8 * j + g) * kTS + 16 * kk + 2 * t;
        mma16816(dw1[j], a1, lds32(xb), lds32(xb + 8));
      }
    }
    __syncthreads();
  }
  // per-CTA partials: weight tiles (one owner per element), column sums reduced
  // over the 8 row groups (xor tree) and then over the 4 warps in order
  float* out = part + (size_t)blockIdx.x * kNParams;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int r0 = 16 * warp + g, c0 = 8 * j + 2 * t;
    out[kOffW2 + r0 * kHid + c0] = dw2[j][0];
    out[kOffW2 + r0 * kHid + c0 + 1] = dw2[j][1];
    out[kOffW2 + (r0 + 8) * kHid + c0] = dw2[j][2];
    out[kOffW2 + (r0 + 8) * kHid + c0 + 1] = dw2[j][3];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r0 = 16 * warp + g, c0 = 8 * j + 2 * t;
    out[kOffW1 + r0 * kIn + c0] = dw1[j][0];
    out[kOffW1 + r0 * kIn + c0 + 1] = dw1[j][1];
    out[kOffW1 + (r0 + 8) * kIn + c0] = dw1[j][2];
    out[kOffW1 + (r0 + 8) * kIn + c0 + 1] = dw1[j][3];
  }
#pragma unroll
  for (int c = 0; c < 16; ++c) {
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      db1[c] += __shfl_xor_sync(0xffffffffu, db1[c], o);
      db2[c] += __shfl_xor_sync(0xffffffffu, db2[c], o);
      dw3[c] += __shfl_xor_sync(0xffffffffu, dw3[c], o);
    }
  }
  db3 += __shfl_xor_sync(0xffffffffu, db3, 4);
  db3 += __shfl_xor_sync(0xffffffffu, db3, 8);
  db3 += __shfl_xor_sync(0xffffffffu, db3, 16);
  if (g == 0) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int col = 8 * (c >> 1) + 2 * t + (c & 1);
      S.red[warp][col] = db1[c];
      S.red[warp][kHid + col] = db2[c];
      S.red[warp][2 * kHid + col] = dw3[c];
    }
    if (t == 0) S.red3[warp] = db3;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 3 * kHid; k += blockDim.x) {
    const float v = ((S.red[0][k] + S.red[1][k]) + S.red[2][k]) + S.red[3][k];
    const int dst = k < kHid ? kOffB1 + k : (k < 2 * kHid ? kOffB2 + k - kHid : kOffW3 + k - 2 * kHid);
    out[dst] = v;
  }
  if (threadIdx.x == 0) out[kOffB3] = ((S.red3[0] + S.red3[1]) + S.red3[2]) + S.red3[3];
}

__global__ void reduce_parts_kernel(const float* __restrict__ part, int nparts, float* __restrict__ grad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kNParams; k += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < nparts; ++c) s += part[(size_t)c * kNParams + k];
    grad[k] = s;
  }
}

// ---------------------------------------------------------------- loss (fp64)

constexpr int kRed = 256;  // threads of the reduction kernels

// Block sums of NV values into part[blockIdx.x * NV + k] (fixed order).
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* part) {
  block_sum<NV>(v);
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) part[(size_t)blockIdx.x * NV + k] = v[k];
}

// Kaporin term, thread per row i: (A g_i)_a for a in P_i (merge of row a of A
// with P_i), quad_i = g_i . (A g_i)_P, log G_ii; partial sums per block.
__global__ void __launch_bounds__(kRed) kaporin_rows_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                                            const int32_t* __restrict__ colind,
                                                            const double* __restrict__ vals,
                                                            const int32_t* __restrict__ trp,
                                                            const int32_t* __restrict__ tci,
                                                            const double* __restrict__ g, double* __restrict__ gag,
                                                            double* part) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int t0 = trp[i], m = trp[i + 1] - t0;
    double quad = 0.0;
    for (int a = 0; a < m; ++a) {
      const int ra = tci[t0 + a];
      double s = 0.0;
      int c = 0;
      for (int k = rowptr[ra]; k < rowptr[ra + 1] && c < m; ++k) {
        const int col = colind[k];
        while (c < m && tci[t0 + c] < col) ++c;
        if (c < m && tci[t0 + c] == col) s += vals[k] * g[t0 + c];
      }
      gag[t0 + a] = s;
      quad += g[t0 + a] * s;
    }
    v[0] += quad;
    v[1] += log(g[t0 + m - 1]);
  }
  block_partials<2>(v, part);
}

// Sum of block partials (one thread per value, blocks in order).
__global__ void sum_parts_kernel(const double* __restrict__ part, int nblocks, int nv, double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k < nv) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * nv + k];
    out[k] = s;
  }
}

// dL_K/dG_e = 2 (A g_i)_a / (n S) - [a == i] 2 / (n G_ii), S = quad / n.
__global__ void kaporin_grad_kernel(int64_t n, const int32_t* __restrict__ trow, const int32_t* __restrict__ tci,
                                    const int32_t* __restrict__ trp, const double* __restrict__ g,
                                    const double* __restrict__ gag, const double* __restrict__ sums, int64_t ntril,
                                    double* __restrict__ dg) {
  const double S = sums[0] / (double)n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ntril; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = trow[e];
    double v = 2.0 * gag[e] / ((double)n * S);
    if (tci[e] == i) v -= 2.0 / ((double)n * g[trp[i + 1] - 1]);
    dg[e] = v;
  }
}

// y = G x (tril CSR with the values g).
__global__ void g_mul_kernel(int64_t n, const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                             const double* __restrict__ g, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = trp[i]; k < trp[i + 1]; ++k) s += g[k] * x[tci[k]];
    y[i] = s;
  }
}

// y = G^T x through the ELL slot map of G^T (src: tril index or -1).
__global__ void gt_mul_kernel(int64_t n, int w, const int32_t* __restrict__ src, const int32_t* __restrict__ col,
                              const double* __restrict__ g, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int m = 0; m < w; ++m) {
      const int e = src[(int64_t)m * n + j];
      if (e >= 0) s += g[e] * x[col[(int64_t)m * n + j]];
    }
    y[j] = s;
  }
}

// y = A x - sub (sub may be null), with the partial sums of y.y and sub.sub.
__global__ void __launch_bounds__(kRed) a_mul_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colind,
                                                     const double* __restrict__ vals, const double* __restrict__ x,
                                                     const double* __restrict__ sub, double* __restrict__ y,
                                                     double* part) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s += vals[k] * x[colind[k]];
    if (sub) {
      s -= sub[i];
      v[1] += sub[i] * sub[i];
    }
    y[i] = s;
    v[0] += s * s;
  }
  block_partials<2>(v, part);
}

// dG_e += scale (u_i Ae_a + GAe_i r_a), scale = 2 lam / (K ||r||^2) from sums.
__global__ void resid_grad_kernel(int64_t ntril, const int32_t* __restrict__ trow, const int32_t* __restrict__ tci,
                                  const double* __restrict__ u, const double* __restrict__ ae,
                                  const double* __restrict__ gae, const double* __restrict__ r,
                                  const double* __restrict__ sums, double coef, double* __restrict__ dg) {
  const double scale = coef / sums[1];  // sums[1] = r.r
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ntril; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = trow[e], a = tci[e];
    dg[e] += scale * (u[i] * ae[a] + gae[i] * r[a]);
  }
}

// dLoss/do = dLoss/dG dG/do.
__global__ void dout_kernel(int64_t ntril, const int32_t* __restrict__ trow, const int32_t* __restrict__ tci,
                            const double* __restrict__ rs64, const float* __restrict__ o,
                            const double* __restrict__ dg, double c0, float* __restrict__ dout) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ntril; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = trow[e], j = tci[e];
    const double d = i == j ? sigmoid_d((double)o[e] + c0) * rs64[i] : rs64[j];
    dout[e] = (float)(dg[e] * d);
  }
}

// fp32 copies of A's values and diagonal and 1 / sqrt(A_ii) in both
// precisions, once per call (the MLP's feature inputs and G's scaling).
__global__ void mlp_inputs_kernel(int64_t n, int64_t nnz, const double* __restrict__ vals,
                                  const double* __restrict__ diag, float* __restrict__ a32, float* __restrict__ d32,
                                  float* __restrict__ rs32, double* __restrict__ rs64) {
  const int64_t m = nnz > n ? nnz : n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    if (k < nnz) a32[k] = (float)vals[k];
    if (k < n) {
      const float d = (float)diag[k];
      d32[k] = d;
      rs32[k] = 1.0f / sqrtf(d);
      rs64[k] = 1.0 / sqrt(diag[k]);
    }
  }
}

// G from the outputs (F5), diagonal entries: thread per row (the diagonal is
// the last tril entry of its row), G_ii = softplus(o + c0) / sqrt(A_ii) in
// fp64, so a zero output gives Jacobi's D^-1/2 to rounding.
__global__ void g_diag_kernel(int64_t n, const int32_t* __restrict__ trp, const double* __restrict__ rs64,
                              const float* __restrict__ o, double c0, double* __restrict__ g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int e = trp[i + 1] - 1;
    g[e] = softplus_d((double)o[e] + c0) * rs64[i];
  }
}

// Off-diagonal entries, thread per entry: G_ij = o / sqrt(A_jj) (the diagonal
// ones are g_diag_kernel's; separate kernels keep warps from running both).
__global__ void g_offdiag_kernel(int64_t ntril, const int32_t* __restrict__ trow, const int32_t* __restrict__ tci,
                                 const double* __restrict__ rs64, const float* __restrict__ o,
                                 double* __restrict__ g) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ntril; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = trow[e], j = tci[e];
    if (i != j) g[e] = (double)o[e] * rs64[j];
  }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int64_t count, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
    const float gk = grad[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  }
}

unsigned blocks_for(int64_t items, int threads = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + threads - 1) / threads, 8192));
}

cg_status mfail(cg_handle* h, cg_status s, const std::string& msg) {
  h->err = msg;
  return s;
}

#define CGM_CUDA(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return mfail((h), e_ == cudaErrorMemoryAllocation ? CG_ERR_OOM : CG_ERR_CUDA,        \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

// Offsets table, row index of every tril entry, work buffers (once per handle).
cg_status mlp_prepare(cg_handle* h) {
  cg_status s = cgi::fsai_pattern(h);
  if (s != CG_OK) return s;
  FsaiData* f = h->fsai;
  if (f->offs) return CG_OK;
  // the distinct offsets j - i: the off-diagonal set and the diagonal (every
  // row has one: fsai_pattern checked it)
  s = cgi::ensure_offsets(h);
  if (s != CG_OK) return s;
  if (h->noffs_all < 0 || h->noffs_all + 1 > kMaxOffs)
    return mfail(h, CG_ERR_INVALID, "learned FSAI: the matrix has more than 9 distinct column offsets");
  std::vector<int32_t> offs(h->offs_all, h->offs_all + h->noffs_all);
  offs.push_back(0);
  std::sort(offs.begin(), offs.end());
  int nts = 0;
  for (int o : offs) nts += o <= 0;
  if (nts > 8) return mfail(h, CG_ERR_INVALID, "learned FSAI: more than 8 offsets in tril(A)");
  CGM_CUDA(h, cudaMalloc(&f->offs, sizeof(int32_t) * kMaxOffs));
  const size_t nv = (size_t)std::max<int64_t>(h->n, 1);
  CGM_CUDA(h, cudaMalloc(&f->a32, sizeof(float) * (size_t)std::max<int64_t>(h->nnz, 1)));
  CGM_CUDA(h, cudaMalloc(&f->d32, sizeof(float) * nv));
  CGM_CUDA(h, cudaMalloc(&f->rs32, sizeof(float) * nv));
  CGM_CUDA(h, cudaMalloc(&f->rs64, sizeof(double) * nv));
  if (!f->mlp_o) CGM_CUDA(h, cudaMalloc(&f->mlp_o, sizeof(float) * (size_t)std::max<int64_t>(f->ntril, 1)));
  f->noffs = (int)offs.size();
  f->ntslots = nts;
  for (int k = 0; k < f->noffs; ++k) f->host_offs[k] = offs[(size_t)k];
  CGM_CUDA(h, cudaMemcpy(f->offs, offs.data(), sizeof(int32_t) * offs.size(), cudaMemcpyHostToDevice));
  return CG_OK;
}

MlpArgs make_args(const cg_handle* h, const float* params) {
  const FsaiData* f = h->fsai;
  MlpArgs M{};
  M.n = h->n;
  M.ntril = f->ntril;
  M.rowptr = h->rowptr;
  M.colind = h->colind;
  M.vals = h->vals;
  M.diag = h->diag;
  M.trow = f->trow;
  M.tci = f->tci;
  M.tsrc = f->tsrc;
  M.params = params;
  M.a32 = f->a32;
  M.d32 = f->d32;
  M.rs32 = f->rs32;
  for (int k = 0; k < kMaxOffs; ++k) M.offs[k] = k < f->noffs ? f->host_offs[k] : 0;
  M.noffs = f->noffs;
  M.ntslots = f->ntslots;
  M.c0 = std::log(std::exp(1.0) - 1.0);
  return M;
}

unsigned mlp_grid(const cg_handle* h, int64_t ntril) {
  const int64_t tiles = (ntril + kTileE - 1) / kTileE;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, 4 * (int64_t)h->sm_count));
}

// Forward (inference) grid: every resident CTA (the feature gathers are
// latency-bound; forward has no per-CTA partials to bound the grid).
unsigned mlp_forward_grid(const cg_handle* h, int64_t ntril) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_forward_kernel, kMlpThreads, 0) != cudaSuccess)
    per_sm = 4;
  const int64_t tiles = (ntril + kTileE - 1) / kTileE;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)std::max(per_sm, 1) * h->sm_count));
}

}  // namespace

extern "C" {

cg_status cg_fsai_load(cg_handle* h, const void* weights_bf16, int64_t bytes) {
  if (!h) return CG_ERR_INVALID;
  if (h->batch) return mfail(h, CG_ERR_INVALID, "cg_fsai_load: batch handle");
  if (!weights_bf16 || bytes != (int64_t)sizeof(uint16_t) * kNParams)
    return mfail(h, CG_ERR_INVALID, "cg_fsai_load: expected " + std::to_string(2 * kNParams) + " bytes of bf16 weights");
  if (h->n == 0) return mfail(h, CG_ERR_INVALID, "cg_fsai_load: empty matrix");
  cg_status s = mlp_prepare(h);
  if (s != CG_OK) return s;
  FsaiData* f = h->fsai;
  // bf16 -> fp32 is exact; the kernels round back to the same bf16 values
  std::vector<float> p32(kNParams);
  const uint16_t* w = static_cast<const uint16_t*>(weights_bf16);
  for (int k = 0; k < kNParams; ++k) {
    const uint32_t bits = (uint32_t)w[k] << 16;
    std::memcpy(&p32[(size_t)k], &bits, sizeof(float));
    if (!std::isfinite(p32[(size_t)k])) return mfail(h, CG_ERR_INVALID, "cg_fsai_load: non-finite weight");
  }
  if (!f->params32) CGM_CUDA(h, cudaMalloc(&f->params32, sizeof(float) * kNParams));
  CGM_CUDA(h, cudaMemcpyAsync(f->params32, p32.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice, h->stream));
  const MlpArgs M = make_args(h, f->params32);
  const int64_t n = h->n, nt = f->ntril;
  mlp_inputs_kernel<<<blocks_for(std::max(n, h->nnz)), 256, 0, h->stream>>>(n, h->nnz, h->vals, h->diag, f->a32,
                                                                            f->d32, f->rs32, f->rs64);
  mlp_forward_kernel<<<mlp_forward_grid(h, nt), kMlpThreads, 0, h->stream>>>(M, f->mlp_o);
  g_diag_kernel<<<blocks_for(n), 256, 0, h->stream>>>(n, f->trp, f->rs64, f->mlp_o, M.c0, f->g);
  g_offdiag_kernel<<<blocks_for(nt), 256, 0, h->stream>>>(nt, f->trow, f->tci, f->rs64, f->mlp_o, f->g);
  CGM_CUDA(h, cudaGetLastError());
  CGM_CUDA(h, cudaStreamSynchronize(h->stream));  // p32 is host memory of this call
  return cgi::fsai_commit(h, 2);
}

cg_status cg_fsai_load_f32(cg_handle* h, const float* weights, int64_t count) {
  if (!h) return CG_ERR_INVALID;
  if (!weights || count != kNParams)
    return mfail(h, CG_ERR_INVALID, "cg_fsai_load_f32: expected " + std::to_string(kNParams) + " fp32 weights");
  // fp32 -> bf16, round to nearest even on the bit pattern: add 0x7FFF plus the
  // lowest kept bit, drop the 16 low bits.  Non-finite inputs are refused before
  // rounding (the carry could turn a NaN payload into an infinity), and a finite
  // value that rounds past the largest bf16 is refused after it.
  std::vector<uint16_t> bits(kNParams);
  for (int k = 0; k < kNParams; ++k) {
    const float w = weights[k];
    if (!std::isfinite(w)) return mfail(h, CG_ERR_INVALID, "cg_fsai_load_f32: non-finite weight " + std::to_string(k));
    uint32_t u;
    std::memcpy(&u, &w, sizeof(u));
    const uint32_t r = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
    if ((r & 0x7F80u) == 0x7F80u)
      return mfail(h, CG_ERR_INVALID, "cg_fsai_load_f32: weight " + std::to_string(k) + " overflows bf16");
    bits[(size_t)k] = (uint16_t)r;
  }
  return cg_fsai_load(h, bits.data(), (int64_t)sizeof(uint16_t) * kNParams);
}

cg_status cg_fsai_loss_grad(cg_handle* h, const float* params, float* grad, const double* resid, int32_t nresid,
                            double lambda, double* loss_out) {
  if (!h) return CG_ERR_INVALID;
  if (h->batch) return mfail(h, CG_ERR_INVALID, "cg_fsai_loss_grad: batch handle");
  if (!params || !grad || nresid < 0 || (nresid > 0 && !resid) || !(lambda >= 0.0) || h->n == 0)
    return mfail(h, CG_ERR_INVALID, "cg_fsai_loss_grad: bad arguments");
  cg_status s = mlp_prepare(h);
  if (s != CG_OK) return s;
  FsaiData* f = h->fsai;
  const int64_t n = h->n, nt = f->ntril;
  const unsigned rb = blocks_for(n, kRed);
  const unsigned mg = mlp_grid(h, nt);
  if (!f->work) {
    CGM_CUDA(h, cudaMalloc(&f->work, sizeof(double) * (6 * (size_t)n + 2 * (size_t)nt)));
    CGM_CUDA(h, cudaMalloc(&f->rpart, sizeof(double) * (8192 * 2 + 16)));
    CGM_CUDA(h, cudaMalloc(&f->dout, sizeof(float) * (size_t)nt));
    CGM_CUDA(h, cudaMalloc(&f->gpart, sizeof(float) * (size_t)(4 * h->sm_count) * kNParams));
    CGM_CUDA(h, cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(SmemB)));
  }
  double* u = f->work;
  double* v = u + n;
  double* e = v + n;
  double* ae = e + n;
  double* gae = ae + n;
  double* gl = gae + n;         // G of the current parameters (tril order)
  double* gag = gl + nt;        // (A g_i)_a, then dLoss/dG
  double* dgv = gag;            // reused: gag is consumed by kaporin_grad_kernel in place
  double* sums = f->rpart + 8192 * 2;  // [0] quad, [1] log-diag, [2] r.r, [3..] residual losses
  const MlpArgs M = make_args(h, params);
  const cudaStream_t st = h->stream;
  mlp_inputs_kernel<<<blocks_for(std::max(n, h->nnz)), 256, 0, st>>>(n, h->nnz, h->vals, h->diag, f->a32, f->d32,
                                                                     f->rs32, f->rs64);
  mlp_forward_kernel<<<mg, kMlpThreads, 0, st>>>(M, f->mlp_o);
  g_diag_kernel<<<blocks_for(n), 256, 0, st>>>(n, f->trp, f->rs64, f->mlp_o, M.c0, gl);
  g_offdiag_kernel<<<blocks_for(nt), 256, 0, st>>>(nt, f->trow, f->tci, f->rs64, f->mlp_o, gl);
  kaporin_rows_kernel<<<rb, kRed, 0, st>>>(n, h->rowptr, h->colind, h->vals, f->trp, f->tci, gl, gag, f->rpart);
  sum_parts_kernel<<<1, 32, 0, st>>>(f->rpart, (int)rb, 2, sums);
  kaporin_grad_kernel<<<blocks_for(nt), 256, 0, st>>>(n, f->trow, f->tci, f->trp, gl, gag, sums, nt, dgv);
  std::vector<double> rloss((size_t)nresid, 0.0);
  for (int k = 0; k < nresid; ++k) {
    const double* r = resid + (size_t)k * n;
    g_mul_kernel<<<blocks_for(n), 256, 0, st>>>(n, f->trp, f->tci, gl, r, u);             // u = G r
    gt_mul_kernel<<<blocks_for(n), 256, 0, st>>>(n, f->gtw, f->gtsrc, f->gtcol, gl, u, v);  // v = G^T u
    a_mul_kernel<<<rb, kRed, 0, st>>>(n, h->rowptr, h->colind, h->vals, v, r, e, f->rpart);  // e = A v - r
    sum_parts_kernel<<<1, 32, 0, st>>>(f->rpart, (int)rb, 2, sums + 2);  // e.e, r.r
    a_mul_kernel<<<rb, kRed, 0, st>>>(n, h->rowptr, h->colind, h->vals, e, nullptr, ae, f->rpart);  // Ae
    g_mul_kernel<<<blocks_for(n), 256, 0, st>>>(n, f->trp, f->tci, gl, ae, gae);                 // G A e
    // dG += 2 lam / (K r.r) (u_i Ae_a + GAe_i r_a)
    resid_grad_kernel<<<blocks_for(nt), 256, 0, st>>>(nt, f->trow, f->tci, u, ae, gae, r, sums + 2,
                                                     2.0 * lambda / nresid, dgv);
    double er[2] = {0.0, 0.0};
    CGM_CUDA(h, cudaMemcpyAsync(er, sums + 2, sizeof(er), cudaMemcpyDeviceToHost, st));
    CGM_CUDA(h, cudaStreamSynchronize(st));  // sums[2..3] are reused by the next vector
    rloss[(size_t)k] = er[0] / er[1];
  }
  dout_kernel<<<blocks_for(nt), 256, 0, st>>>(nt, f->trow, f->tci, f->rs64, f->mlp_o, dgv, M.c0, f->dout);
  mlp_backward_kernel<<<mg, kMlpThreads, sizeof(SmemB), st>>>(M, f->dout, f->gpart);
  reduce_parts_kernel<<<blocks_for(kNParams), 256, 0, st>>>(f->gpart, (int)mg, grad);
  CGM_CUDA(h, cudaGetLastError());
  double hs[2] = {0.0, 0.0};
  CGM_CUDA(h, cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, st));
  CGM_CUDA(h, cudaStreamSynchronize(st));
  double loss = std::log(hs[0] / (double)n) - 2.0 / (double)n * hs[1];
  if (nresid > 0) {
    double lr = 0.0;
    for (double x : rloss) lr += x;
    loss += lambda * lr / nresid;
  }
  if (loss_out) *loss_out = loss;
  if (!std::isfinite(loss)) return mfail(h, CG_ERR_NUMERIC, "cg_fsai_loss_grad: non-finite loss");
  return CG_OK;
}

cg_status cg_adam_step(float* params, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                       float beta2, float eps, int32_t step, void* stream) {
  if (!params || !grad || !m || !v || count <= 0 || step < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return CG_ERR_INVALID;
  const float c1 = 1.0f - std::pow(beta1, (float)step), c2 = 1.0f - std::pow(beta2, (float)step);
  adam_kernel<<<blocks_for(count), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(params, grad, m, v, count, lr,
                                                                                    beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

}  // extern "C"
