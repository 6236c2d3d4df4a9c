// The decoder F_de (Eq. 4) of PGS_DECODE_BF16 / BF16_1PASS on the tensor
// cores, as stages shared by the forward kernel (decode + projection) and the
// backward kernel (which recomputes the forward bit for bit).
//
// Precision per output head (see k_decode_tc.cu for the reasons):
//   layer 1  D1[128 x 32]  = X . W1^T            three-piece BF16 split of X and W1,
//                                                 six products (FP32-accurate)
//   layer 2  colour block   D2[:, 0..31]  = bf16(H) . bf16(W2_colour)^T   one pass
//            shape block    D2[:, 32..111] = H . W2_shape^T                 six products
// A three-piece split x = p0 + p1 + p2 (BF16 each) is exact for FP32 x; the
// products p_i q_j with i + j <= 2 leave out terms below 2^-24 |x q|.  The
// one-pass study form keeps only p0 q0 everywhere.
//
// Layouts: operands in the no-swizzle K-major core-matrix layout; layer-2
// column n holds Eq. 4's output l2_out(n): colour of Gaussian n / 3 (channel
// n % 3) for n < 30, then per Gaussian j the 8 columns 32 + 8 j + (opacity,
// scale x3, rotation x4).  TMEM: D1 at column 0, D2 at column 32.
#pragma once
#include <cuda_bf16.h>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"
#include "pgs_project.cuh"
#include "pgs_tc.cuh"

namespace pgs {
namespace tc {

constexpr int kRows = 128;
constexpr int kK1 = 48, kN1 = 32;           // layer 1: K padded from 35 (or 36), N = hidden
constexpr int kK2 = 32, kN2 = 112;          // layer 2: K = hidden, N = colour block 32 + shape block 80
constexpr int kShape0 = 32, kNShape = 80, kPerShape = 8;
constexpr uint32_t kD2Col = 32;

struct DecSmem {
  __nv_bfloat16 A1[3][kRows * kK1];         // X pieces   3 x 12288 B
  __nv_bfloat16 B1[3][kN1 * kK1];           // W1 pieces  3 x  3072 B
  __nv_bfloat16 A2[3][kRows * kK2];         // H pieces   3 x  8192 B
  __nv_bfloat16 B2[3][kN2 * kK2];           // W2 pieces  3 x  7168 B, rows in layer-2 column order
  float b1[kN1];
  float b2p[kN2];
  unsigned long long mbar;
  uint32_t tmem_base;
};

// layer-2 column n -> index in Eq. 4's blocked output [opacity x10 | colour x30 |
// scale x30 | quat x40], or -1 (padding)
__host__ __device__ inline int l2_out(int n) {
  if (n < 30) return 10 + n;
  if (n < kShape0) return -1;
  const int m = n - kShape0, j = m / kPerShape, t = m % kPerShape;
  if (t == 0) return j;
  if (t <= 3) return 40 + 3 * j + (t - 1);
  return 70 + 4 * j + (t - 4);
}

__device__ __forceinline__ void put_bf16(__nv_bfloat16* tile, uint32_t off, __nv_bfloat16 v) {
  *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(tile) + off) = v;
}
__device__ __forceinline__ void put_bf16x2(__nv_bfloat16* tile, uint32_t off, __nv_bfloat16 a, __nv_bfloat16 b) {
  *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<char*>(tile) + off) = __halves2bfloat162(a, b);
}

// decoder weights -> BF16 operand pieces (zero padded); biases stay FP32 (all threads)
__device__ __forceinline__ void dec_stage_weights(DecSmem& sm, const pgs_mlp_ptrs& Wt, int in_dim, int pieces) {
  for (int t = threadIdx.x; t < kN1 * kK1; t += blockDim.x) {
    const int n = t / kK1, k = t % kK1;
    const float w = k < in_dim ? Wt.W1[n * in_dim + k] : 0.f;
    __nv_bfloat16 p[3];
    split3(w, p[0], p[1], p[2]);
    for (int i = 0; i < pieces; ++i) put_bf16(sm.B1[i], kmaj_off(n, k, kK1), p[i]);
  }
  for (int t = threadIdx.x; t < kN2 * kK2; t += blockDim.x) {
    const int n = t / kK2, k = t % kK2;
    const int o = l2_out(n);
    const float w = o >= 0 ? Wt.W2[o * kHidden + k] : 0.f;
    __nv_bfloat16 p[3];
    split3(w, p[0], p[1], p[2]);
    for (int i = 0; i < pieces; ++i) put_bf16(sm.B2[i], kmaj_off(n, k, kK2), p[i]);
  }
  if (threadIdx.x < kN1) sm.b1[threadIdx.x] = Wt.b1[threadIdx.x];
  for (int t = threadIdx.x; t < kN2; t += blockDim.x) {
    const int o = l2_out(t);
    sm.b2p[t] = o >= 0 ? Wt.b2[o] : 0.f;
  }
}

// layer-1 operand row `row` (pieces), X (FP32) left in X (zero for a row past n_rows)
__device__ __forceinline__ void dec_stage_x(DecSmem& sm, const BatchDev& b, const pgs_anchor_ptrs& A,
                                            const uint32_t* __restrict__ rows, long long r, long long n_rows, int row,
                                            int pieces, float (&X)[kMaxIn]) {
  const int in_dim = b.p.in_dim;
#pragma unroll
  for (int k = 0; k < kMaxIn; ++k) X[k] = 0.f;
  if (r < n_rows) {
    const uint32_t rw = rows[r];
    decoder_input(A, b.v[rw >> 27], rw & ((1u << 27) - 1), in_dim, X);
  }
#pragma unroll
  for (int k = 0; k < kK1; k += 2) {
    const float x0 = (k < kMaxIn && k < in_dim) ? X[k < kMaxIn ? k : 0] : 0.f;
    const float x1 = (k + 1 < kMaxIn && k + 1 < in_dim) ? X[k + 1 < kMaxIn ? k + 1 : 0] : 0.f;
    __nv_bfloat16 p0[3], p1[3];
    split3(x0, p0[0], p0[1], p0[2]);
    split3(x1, p1[0], p1[1], p1[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (i < pieces) put_bf16x2(sm.A1[i], kmaj_off(row, k, kK1), p0[i], p1[i]);
  }
}

// layer-1 MMAs (one thread): D1 = X . W1^T, split products smallest first
__device__ __forceinline__ void dec_issue_layer1(DecSmem& sm, uint32_t tmem, bool split) {
  constexpr uint32_t kIdesc1 = make_idesc(kRows, kN1);
  uint32_t acc = 0;
#pragma unroll
  for (int t = 0; t < kSplitProducts; ++t) {
    if (!split && t != kSplitProducts - 1) continue;
    int i, j;
    split_product(t, i, j);
#pragma unroll
    for (int kk = 0; kk < kK1 / 16; ++kk) {
      mma_bf16(tmem, kmaj_desc(smem_u32(sm.A1[i]), kK1, 0, kk), kmaj_desc(smem_u32(sm.B1[j]), kK1, 0, kk), kIdesc1,
               acc);
      acc = 1;
    }
  }
}

// hidden layer of row `row`: H = ReLU(D1 + b1) into h (FP32) and the layer-2 operand pieces
__device__ __forceinline__ void dec_stage_h(DecSmem& sm, uint32_t tlane, int row, int pieces, float (&h)[kHidden]) {
  tmem_ld32(tlane, h);
#pragma unroll
  for (int k = 0; k < kK2; k += 2) {
    h[k] = fmaxf(h[k] + sm.b1[k], 0.f);
    h[k + 1] = fmaxf(h[k + 1] + sm.b1[k + 1], 0.f);
    __nv_bfloat16 p0[3], p1[3];
    split3(h[k], p0[0], p0[1], p0[2]);
    split3(h[k + 1], p1[0], p1[1], p1[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (i < pieces) put_bf16x2(sm.A2[i], kmaj_off(row, k, kK2), p0[i], p1[i]);
  }
}

// layer-2 MMAs (one thread): colour block one BF16 pass, shape block the split products
__device__ __forceinline__ void dec_issue_layer2(DecSmem& sm, uint32_t tmem, bool split) {
  constexpr uint32_t kIdescC = make_idesc(kRows, 32), kIdescS = make_idesc(kRows, kNShape);
#pragma unroll
  for (int kk = 0; kk < kK2 / 16; ++kk)
    mma_bf16(tmem + kD2Col, kmaj_desc(smem_u32(sm.A2[0]), kK2, 0, kk), kmaj_desc(smem_u32(sm.B2[0]), kK2, 0, kk),
             kIdescC, kk > 0 ? 1u : 0u);
  uint32_t acc = 0;
#pragma unroll
  for (int t = 0; t < kSplitProducts; ++t) {
    if (!split && t != kSplitProducts - 1) continue;
    int i, j;
    split_product(t, i, j);
#pragma unroll
    for (int kk = 0; kk < kK2 / 16; ++kk) {
      mma_bf16(tmem + kD2Col + kShape0, kmaj_desc(smem_u32(sm.A2[i]), kK2, 0, kk),
               kmaj_desc(smem_u32(sm.B2[j]), kK2, kShape0, kk), kIdescS, acc);
      acc = 1;
    }
  }
}

// the colour columns of part P's Gaussians (4P .. 4P + nG - 1): 3 nG values
template <int P, int NG>
__device__ __forceinline__ void dec_load_colour(uint32_t tlane, float (&cz)[3 * NG]) {
  float c32[32];
  tmem_ld32(tlane + kD2Col, c32);
#pragma unroll
  for (int i = 0; i < 3 * NG; ++i) cz[i] = c32[12 * P + i];
}

// Eq. 4's 11 outputs (opacity, colour x3, scale x3, quaternion x4) of Gaussian
// j from its colour values c[3] and shape-block values s8[8], biases added
__device__ __forceinline__ void dec_outputs(const float* b2p, int j, const float* c, const float* s8, float (&z)[11]) {
  const int s0 = kShape0 + kPerShape * j;
  z[0] = s8[0] + b2p[s0];
#pragma unroll
  for (int q = 0; q < 3; ++q) z[1 + q] = c[q] + b2p[3 * j + q];
#pragma unroll
  for (int q = 0; q < 3; ++q) z[4 + q] = s8[1 + q] + b2p[s0 + 1 + q];
#pragma unroll
  for (int q = 0; q < 4; ++q) z[7 + q] = s8[4 + q] + b2p[s0 + 4 + q];
}

}  // namespace tc
}  // namespace pgs
