// Backward of the tensor-core decoder (PGS_DECODE_BF16) on the tensor cores:
// the decoder of Eq. 4 is shared by every view, so its gradient flows from all
// visible (view, anchor) rows of the batch.
//
// One CTA of 384 threads takes 128 rows at a time:
//  1. the forward is recomputed with the forward kernel's own stages and MMAs
//     (same operands, same products, same order: the same H and Z bits);
//  2. per Gaussian (warps of the three epilogue parts, as in the forward): the
//     activations and the projection backward of its 13 gradient-record
//     entries give dZ (11 outputs), the per-anchor gradients of the offsets,
//     the scaling factor and the position; dZ goes to shared memory as two
//     BF16 pieces (dZ = d0 + d1 to 2^-16) and, in FP32, to the row scratch of
//     the weight gradients;
//  3. dH = dZ . W2 on the tensor cores: over the colour block with the BF16
//     weight the forward multiplied (its one pass: the gradient passes
//     straight through that rounding), over the shape block with W2 in two
//     pieces; products d1 w0 + d0 w1 + d0 w0, FP32 accumulation in TMEM;
//  4. dH' = dH . [H > 0] (row threads) -> scratch and two BF16 pieces;
//  5. dX = dH' . W1 on the tensor cores (two-piece operands, three products);
//     the feature part is the anchor feature gradient, the view-direction
//     part goes to the anchor position through d(unit direction)/dx.
// Every MMA wait is bounded as in the forward.
//
// The decoder's weight gradients (k_mlp_wgrad_tc) are a reduction over all
// rows of the batch, done on the tensor cores from the FP32 row scratch, 128
// rows (the MMA's K) at a time, accumulated in TMEM across a CTA's chunks:
//   dW2: D[o][n] = sum_r dZ[r][o] B[n][r], A = dZ^T in two pieces (two MMAs),
//        B = [H0 | H1 | 1]: dW2[o][h] = D[o][h] + D[o][32 + h] for the shape
//        heads and D[o][h] alone for the colour heads, whose forward took the
//        BF16-rounded H0 (the straight-through gradient of that rounding);
//        db2[o] = D[o][64];
//   dW1: D[m][n] = sum_r A[m][r] B[n][r], A = [dH'0 | dH'1]^T stacked along M,
//        B = [X0 | X1 | 1]: dW1[h][i] = D[h][i] + D[h][36 + i] + D[32 + h][i],
//        db1[h] = D[h][72] + D[32 + h][72].
// Each CTA writes its sums to a partial row; k_mlp_wgrad_final adds the
// partials in CTA order (deterministic).
#include <algorithm>

#include "pgs_backward.cuh"
#include "pgs_decode_tc.cuh"

namespace pgs {

using namespace tc;

namespace {

constexpr int kBwdThreads = 384;
constexpr uint32_t kBwdTmemCols = 256;
constexpr uint32_t kDHCol = 144, kDXCol = 176;     // after D1 (0..31) and D2 (32..143)
constexpr int kDXN = 48;                           // dX columns (inputs padded to 48)

struct BwdSmem {
  DecSmem f;
  __nv_bfloat16 dZ[2][kRows * kN2];       // dZ pieces [128 rows x 112 layer-2 columns], K-major   2 x 28672 B
  __nv_bfloat16 W2t[2][kHidden * kN2];    // W2 as the B operand of dH: [32 hidden x 112 columns]  2 x  7168 B
  __nv_bfloat16 dHs[2][kRows * kK2];      // dH' pieces [128 x 32]                                 2 x  8192 B
  __nv_bfloat16 W1t[2][kK1 * kK2];        // W1 as the B operand of dX: [48 inputs x 32 hidden]    2 x  3072 B
};

// backward of part P's Gaussians of one row: dZ into shared memory (and the
// scratch), per-anchor gradients; a row past n_rows writes zeros
template <int P>
__device__ __forceinline__ void bwd_epilogue(const BatchDev& b, const pgs_anchor_ptrs& A, BwdSmem& sm, uint32_t tlane,
                                             int erow, bool valid, int vi, long long a, long long r,
                                             const float* __restrict__ grad, pgs_param_grad_ptrs out,
                                             float* __restrict__ sc_dZ, bool& bad) {
  constexpr int nG = P == 2 ? 2 : 4;
  float cz[3 * nG];
  dec_load_colour<P, nG>(tlane, cz);
  float l[3] = {1.f, 1.f, 1.f}, xa[3] = {0.f, 0.f, 0.f};
  if (valid) {
    l[0] = expf(A.log_l[3 * a]); l[1] = expf(A.log_l[3 * a + 1]); l[2] = expf(A.log_l[3 * a + 2]);
    xa[0] = A.x[3 * a]; xa[1] = A.x[3 * a + 1]; xa[2] = A.x[3 * a + 2];
  }
  float dl[3] = {0.f, 0.f, 0.f}, dxa[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int u2 = 0; u2 < nG / 2; ++u2) {
    float sz[16];
    tmem_ld16(tlane + kD2Col + kShape0 + 32 * P + 16 * u2, sz);
#pragma unroll 1
    for (int w = 0; w < 2; ++w) {
      const int u = 2 * u2 + w, j = 4 * P + u;
      float dz[11];
#pragma unroll
      for (int t = 0; t < 11; ++t) dz[t] = 0.f;
      float gr[13];
      if (valid && load_grad(grad, r * kNOff + j, gr)) {
        float c3[3], s8[8];          // this Gaussian's columns (selected, so the arrays stay in registers)
#pragma unroll
        for (int t = 0; t < 3; ++t) c3[t] = w ? cz[3 * (2 * u2 + 1) + t] : cz[3 * (2 * u2) + t];
#pragma unroll
        for (int t = 0; t < 8; ++t) s8[t] = w ? sz[8 + t] : sz[t];
        float z[11];
        dec_outputs(sm.f.b2p, j, c3, s8, z);
        const float op = sigm(z[0]);
        const float col[3] = {sigm(z[1]), sigm(z[2]), sigm(z[3])};
        const float sgs[3] = {sigm(z[4]), sigm(z[5]), sigm(z[6])};
        const float s[3] = {l[0] * sgs[0], l[1] * sgs[1], l[2] * sgs[2]};
        const float qr[4] = {z[7], z[8], z[9], z[10]};
        const float qn = sqrtf(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
        float q[4] = {1.f, 0.f, 0.f, 0.f};
        if (qn >= 1e-12f) { const float iq = 1.f / qn; for (int t = 0; t < 4; ++t) q[t] = qr[t] * iq; }
        const float* O = A.offsets + (a * kNOff + j) * 3;
        const float mu[3] = {xa[0] + O[0] * l[0], xa[1] + O[1] * l[1], xa[2] + O[2] * l[2]};
        ProjGrad pg;
        project_backward(b, b.v[vi], mu, s, q, gr, pg);
        float dq[4];
        quat_norm_backward(qr, qn, pg.dq, dq);
        dz[0] = pg.dop * op * (1.f - op);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          dz[1 + t] = pg.dcol[t] * col[t] * (1.f - col[t]);
          dz[4 + t] = pg.ds[t] * l[t] * sgs[t] * (1.f - sgs[t]);
          dl[t] += pg.ds[t] * sgs[t] + pg.dmu[t] * O[t];
          dxa[t] += pg.dmu[t];
          add_if(out.offsets ? out.offsets + (a * kNOff + j) * 3 + t : nullptr, pg.dmu[t] * l[t]);
          bad |= !isfinite(pg.dmu[t]) || !isfinite(pg.ds[t]);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) dz[7 + t] = dq[t];
      }
      // dZ in layer-2 column order: colour at 3 j + c, shape block at 32 + 8 j + (opacity, scale, rotation)
      const int s0 = kShape0 + kPerShape * j;
      const int col_of[11] = {s0, 3 * j, 3 * j + 1, 3 * j + 2, s0 + 1, s0 + 2, s0 + 3, s0 + 4, s0 + 5, s0 + 6, s0 + 7};
      const int out_of[11] = {j, 10 + 3 * j, 11 + 3 * j, 12 + 3 * j, 40 + 3 * j, 41 + 3 * j, 42 + 3 * j,
                              70 + 4 * j, 71 + 4 * j, 72 + 4 * j, 73 + 4 * j};
#pragma unroll
      for (int t = 0; t < 11; ++t) {
        __nv_bfloat16 p0, p1, p2;
        split3(dz[t], p0, p1, p2);
        put_bf16(sm.dZ[0], kmaj_off(erow, col_of[t], kN2), p0);
        put_bf16(sm.dZ[1], kmaj_off(erow, col_of[t], kN2), p1);
        if (valid) sc_dZ[sc_at(r, out_of[t], kOut)] = dz[t];
      }
    }
  }
  if (valid) {
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      add_if(out.x ? out.x + 3 * a + t : nullptr, dxa[t]);
      add_if(out.log_l ? out.log_l + 3 * a + t : nullptr, dl[t] * l[t]);
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(kBwdThreads, 1) k_decode_bwd_tc(
    const __grid_constant__ BatchDev b, pgs_anchor_ptrs A, pgs_mlp_ptrs Wt, const uint32_t* __restrict__ rows,
    const long long* __restrict__ n_rows_p, long long cap, const float* __restrict__ grad, pgs_param_grad_ptrs out,
    float* __restrict__ sc_dZ, float* __restrict__ sc_H, float* __restrict__ sc_dH, float* __restrict__ sc_X,
    uint32_t* err) {
  extern __shared__ unsigned char smem_raw[];
  BwdSmem& sm = *reinterpret_cast<BwdSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool row_thread = tid < kRows;
  const int erow = (warp & 3) * 32 + (tid & 31);
  const int epart = warp >> 2;
  const int in_dim = b.p.in_dim;
  dec_stage_weights(sm.f, Wt, in_dim, 3);
  // the backward's B operands (two pieces; the colour columns only the BF16 weight the forward used)
  for (int t = tid; t < kHidden * kN2; t += kBwdThreads) {
    const int h = t / kN2, c = t % kN2;
    const int o = l2_out(c);
    const float w = o >= 0 ? Wt.W2[o * kHidden + h] : 0.f;
    __nv_bfloat16 p0, p1, p2;
    split3(w, p0, p1, p2);
    put_bf16(sm.W2t[0], kmaj_off(h, c, kN2), p0);
    put_bf16(sm.W2t[1], kmaj_off(h, c, kN2), c < kShape0 ? __float2bfloat16_rn(0.f) : p1);
  }
  for (int t = tid; t < kK1 * kK2; t += kBwdThreads) {
    const int i = t / kK2, h = t % kK2;
    const float w = i < in_dim ? Wt.W1[h * in_dim + i] : 0.f;
    __nv_bfloat16 p0, p1, p2;
    split3(w, p0, p1, p2);
    put_bf16(sm.W1t[0], kmaj_off(i, h, kK2), p0);
    put_bf16(sm.W1t[1], kmaj_off(i, h, kK2), p1);
  }
  // the padding columns 30, 31 of the dZ tiles are never written by the epilogue: zero them once
  for (int t = tid; t < kRows * 2; t += kBwdThreads) {
    const int row = t >> 1, c = 30 + (t & 1);
    put_bf16(sm.dZ[0], kmaj_off(row, c, kN2), __float2bfloat16_rn(0.f));
    put_bf16(sm.dZ[1], kmaj_off(row, c, kN2), __float2bfloat16_rn(0.f));
  }
  const uint32_t mbar = smem_u32(&sm.f.mbar);
  if (tid == 0) mbar_init(mbar);
  if (warp == 0) tmem_alloc(&sm.f.tmem_base, kBwdTmemCols);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.f.tmem_base;
  const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  const long long n_rows = min(*n_rows_p, cap);
  const long long n_tiles = (n_rows + kRows - 1) / kRows;
  uint32_t phase = 0;
  bool timed_out = false, bad = false;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long rr = tile * kRows + tid;            // row of a row thread
    uint32_t relu_mask = 0;
    if (row_thread) {
      float X[kMaxIn];
      dec_stage_x(sm.f, b, A, rows, rr, n_rows, tid, 3, X);
      if (rr < n_rows) {
#pragma unroll
        for (int k = 0; k < kMaxIn; ++k)
          if (k < in_dim) sc_X[sc_at(rr, k, kMaxIn)] = X[k];
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      dec_issue_layer1(sm.f, tmem, true);
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase))) { timed_out = true; break; }
    phase ^= 1u;
    fence_after();
    if (row_thread) {
      float h[kHidden];
      dec_stage_h(sm.f, tlane, tid, 3, h);
#pragma unroll
      for (int k = 0; k < kHidden; ++k) relu_mask |= (h[k] > 0.f ? 1u : 0u) << k;
      if (rr < n_rows) {
#pragma unroll
        for (int k = 0; k < kHidden; ++k) sc_H[sc_at(rr, k, kHidden)] = h[k];
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      dec_issue_layer2(sm.f, tmem, true);
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase))) { timed_out = true; break; }
    phase ^= 1u;
    fence_after();
    // per-Gaussian backward of this thread's part
    {
      const long long r = tile * kRows + erow;
      const bool valid = r < n_rows;
      int vi = 0;
      long long a = 0;
      if (valid) {
        const uint32_t rw = rows[r];
        vi = rw >> 27;
        a = rw & ((1u << 27) - 1);
      }
      if (epart == 0) bwd_epilogue<0>(b, A, sm, tlane, erow, valid, vi, a, r, grad, out, sc_dZ, bad);
      else if (epart == 1) bwd_epilogue<1>(b, A, sm, tlane, erow, valid, vi, a, r, grad, out, sc_dZ, bad);
      else bwd_epilogue<2>(b, A, sm, tlane, erow, valid, vi, a, r, grad, out, sc_dZ, bad);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      // dH = dZ . W2: colour block (k-steps 0, 1) with the BF16 weight, shape block (k-steps 2..6) with two pieces
      fence_after();
      constexpr uint32_t kIdH = make_idesc(kRows, kHidden);
      const uint32_t dz0 = smem_u32(sm.dZ[0]), dz1 = smem_u32(sm.dZ[1]);
      const uint32_t w0 = smem_u32(sm.W2t[0]), w1 = smem_u32(sm.W2t[1]);
      uint32_t acc = 0;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        mma_bf16(tmem + kDHCol, kmaj_desc(dz1, kN2, 0, kk), kmaj_desc(w0, kN2, 0, kk), kIdH, acc);
        acc = 1;
        mma_bf16(tmem + kDHCol, kmaj_desc(dz0, kN2, 0, kk), kmaj_desc(w0, kN2, 0, kk), kIdH, 1u);
      }
#pragma unroll
      for (int kk = 2; kk < kN2 / 16; ++kk) {
        mma_bf16(tmem + kDHCol, kmaj_desc(dz1, kN2, 0, kk), kmaj_desc(w0, kN2, 0, kk), kIdH, 1u);
        mma_bf16(tmem + kDHCol, kmaj_desc(dz0, kN2, 0, kk), kmaj_desc(w1, kN2, 0, kk), kIdH, 1u);
        mma_bf16(tmem + kDHCol, kmaj_desc(dz0, kN2, 0, kk), kmaj_desc(w0, kN2, 0, kk), kIdH, 1u);
      }
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase))) { timed_out = true; break; }
    phase ^= 1u;
    fence_after();
    if (row_thread) {
      float dh[kHidden];
      tmem_ld32(tlane + kDHCol, dh);
#pragma unroll
      for (int k = 0; k < kHidden; k += 2) {
        const float g0 = (relu_mask >> k) & 1u ? dh[k] : 0.f;
        const float g1 = (relu_mask >> (k + 1)) & 1u ? dh[k + 1] : 0.f;
        if (rr < n_rows) {
          sc_dH[sc_at(rr, k, kHidden)] = g0;
          sc_dH[sc_at(rr, k + 1, kHidden)] = g1;
        }
        __nv_bfloat16 a0, a1, a2, c0, c1, c2;
        split3(g0, a0, a1, a2);
        split3(g1, c0, c1, c2);
        put_bf16x2(sm.dHs[0], kmaj_off(tid, k, kK2), a0, c0);
        put_bf16x2(sm.dHs[1], kmaj_off(tid, k, kK2), a1, c1);
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      // dX = dH' . W1 (two-piece operands)
      fence_after();
      constexpr uint32_t kIdX = make_idesc(kRows, kDXN);
      const uint32_t h0 = smem_u32(sm.dHs[0]), h1 = smem_u32(sm.dHs[1]);
      const uint32_t w0 = smem_u32(sm.W1t[0]), w1 = smem_u32(sm.W1t[1]);
      uint32_t acc = 0;
#pragma unroll
      for (int kk = 0; kk < kK2 / 16; ++kk) {
        mma_bf16(tmem + kDXCol, kmaj_desc(h1, kK2, 0, kk), kmaj_desc(w0, kK2, 0, kk), kIdX, acc);
        acc = 1;
        mma_bf16(tmem + kDXCol, kmaj_desc(h0, kK2, 0, kk), kmaj_desc(w1, kK2, 0, kk), kIdX, 1u);
        mma_bf16(tmem + kDXCol, kmaj_desc(h0, kK2, 0, kk), kmaj_desc(w0, kK2, 0, kk), kIdX, 1u);
      }
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase))) { timed_out = true; break; }
    phase ^= 1u;
    fence_after();
    if (row_thread) {
      float dx[32], dx2[16];
      tmem_ld32(tlane + kDXCol, dx);
      tmem_ld16(tlane + kDXCol + 32, dx2);
      if (rr < n_rows) {
        const uint32_t rw = rows[rr];
        const ViewDev& v = b.v[rw >> 27];
        const long long a = rw & ((1u << 27) - 1);
#pragma unroll
        for (int k = 0; k < kFeat; ++k) add_if(out.feat ? out.feat + a * kFeat + k : nullptr, dx[k]);
        // unit view direction dir = (x - o)/|x - o|: d dir / dx = (I - dir dir^T) / |x - o|
        const float ddx = A.x[3 * a] - v.center[0], ddy = A.x[3 * a + 1] - v.center[1], ddz = A.x[3 * a + 2] - v.center[2];
        const float dist = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
        const float idist = 1.f / dist;
        const float d0 = ddx * idist, d1 = ddy * idist, d2 = ddz * idist;
        const float dd = d0 * dx2[0] + d1 * dx2[1] + d2 * dx2[2];
        float g[3] = {(dx2[0] - d0 * dd) * idist, (dx2[1] - d1 * dd) * idist, (dx2[2] - d2 * dd) * idist};
        if (in_dim == 36) { g[0] += dx2[3] * d0; g[1] += dx2[3] * d1; g[2] += dx2[3] * d2; }
#pragma unroll
        for (int t = 0; t < 3; ++t) add_if(out.x ? out.x + 3 * a + t : nullptr, g[t]);
      }
    }
    fence_before();
    __syncthreads();
  }
  if (bad) set_flag(err, kFlagNonfinite);
  if (timed_out) {
    if (tid == 0) set_flag(err, kFlagTimeout);
    (void)mbar_wait(mbar, phase);   // let the MMA in flight finish before the memory is released
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kBwdTmemCols);
  }
}

// ---------------------------------------------------------------- weight gradients on the tensor cores
namespace {

constexpr int kWgThreads = 384;
constexpr int kWgK = 128;                     // rows per chunk (the MMA's K)
constexpr int kWgN = 80;                      // B columns: [piece 0 | piece 1 | ones | zero]
constexpr uint32_t kWgTmemCols = 256;         // dW2 accumulator at column 0, dW1 at column 128
constexpr uint32_t kWgW1Col = 128;

struct WgSmem {
  __nv_bfloat16 Az[2][128 * kWgK];            // dZ^T pieces [o x r]        2 x 32768 B
  __nv_bfloat16 Ad[128 * kWgK];               // [dH'0^T ; dH'1^T ; 0]       32768 B
  __nv_bfloat16 Bh[kWgN * kWgK];              // [H0 | H1 | 1 | 0]           20480 B
  __nv_bfloat16 Bx[kWgN * kWgK];              // [X0 | X1 | 1 | 0]           20480 B
  float red[32][kWgN];                        // dW1 rows of piece 1 (warp 1 -> warp 0)
  unsigned long long mbar;
  uint32_t tmem_base;
};

// 8 consecutive scratch rows (r0 .. r0 + 7, one 16-byte core-matrix row) of feature f; zeros past n
__device__ __forceinline__ void wg_load8(const float* __restrict__ sc, long long r0, int f, int width, long long n,
                                         float (&v)[8]) {
  if (r0 + 8 <= n) {
    const float4* p = reinterpret_cast<const float4*>(sc + sc_at(r0, f, width));
    const float4 a = p[0], c = p[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = c.x; v[5] = c.y; v[6] = c.z; v[7] = c.w;
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = r0 + i < n ? sc[sc_at(r0 + i, f, width)] : 0.f;
  }
}

// BF16 piece 0 of 8 values as one 16-byte core-matrix row (t1: piece 1 as another)
__device__ __forceinline__ void wg_store8(__nv_bfloat16* t0, __nv_bfloat16* t1, uint32_t off, const float (&v)[8]) {
  __nv_bfloat162 h0[4], h1[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat16 a0, a1, a2, b0, b1, b2;
    split3(v[2 * i], a0, a1, a2);
    split3(v[2 * i + 1], b0, b1, b2);
    h0[i] = __halves2bfloat162(a0, b0);
    h1[i] = __halves2bfloat162(a1, b1);
  }
  *reinterpret_cast<uint4*>(reinterpret_cast<char*>(t0) + off) = *reinterpret_cast<const uint4*>(h0);
  if (t1) *reinterpret_cast<uint4*>(reinterpret_cast<char*>(t1) + off) = *reinterpret_cast<const uint4*>(h1);
}

__device__ __forceinline__ void wg_fill8(__nv_bfloat16* t, uint32_t off, float x) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, x);
  const uint32_t u = *reinterpret_cast<const uint32_t*>(&h);
  *reinterpret_cast<uint4*>(reinterpret_cast<char*>(t) + off) = make_uint4(u, u, u, u);
}

}  // namespace

__global__ void __launch_bounds__(kWgThreads, 1) k_mlp_wgrad_tc(const float* __restrict__ sc_dZ,
                                                               const float* __restrict__ sc_H,
                                                               const float* __restrict__ sc_dH,
                                                               const float* __restrict__ sc_X,
                                                               const long long* __restrict__ n_rows_p, long long cap,
                                                               int in_dim, float* __restrict__ partials,
                                                               uint32_t* err) {
  extern __shared__ unsigned char smem_raw[];
  WgSmem& sm = *reinterpret_cast<WgSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kGroups = kWgK / 8;                       // 16 core-matrix rows along K
  // constant parts: zero rows, the ones rows
  for (int t = tid; t < 128 * kGroups; t += kWgThreads) {
    const int m = t / kGroups, g = t % kGroups;
    const uint32_t off = kmaj_off(m, 8 * g, kWgK);
    if (m >= kOut) { wg_fill8(sm.Az[0], off, 0.f); wg_fill8(sm.Az[1], off, 0.f); }
    if (m >= 2 * kHidden) wg_fill8(sm.Ad, off, 0.f);
    if (m >= 2 * kHidden && m < kWgN) wg_fill8(sm.Bh, off, m == 2 * kHidden ? 1.f : 0.f);
    if (m < kWgN && (m >= 2 * kMaxIn || (m % kMaxIn) >= in_dim))
      wg_fill8(sm.Bx, off, m == 2 * kMaxIn ? 1.f : 0.f);
  }
  const uint32_t mbar = smem_u32(&sm.mbar);
  if (tid == 0) mbar_init(mbar);
  if (warp == 0) tmem_alloc(&sm.tmem_base, kWgTmemCols);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.tmem_base;
  const long long n = min(*n_rows_p, cap);
  const long long n_chunks = (n + kWgK - 1) / kWgK;
  uint32_t phase = 0, acc = 0;
  bool timed_out = false;
  for (long long ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const long long r0 = ch * kWgK;
    for (int t = tid; t < kOut * kGroups; t += kWgThreads) {         // dZ^T
      const int o = t / kGroups, g = t % kGroups;
      float v[8];
      wg_load8(sc_dZ, r0 + 8 * g, o, kOut, n, v);
      wg_store8(sm.Az[0], sm.Az[1], kmaj_off(o, 8 * g, kWgK), v);
    }
    for (int t = tid; t < kHidden * kGroups; t += kWgThreads) {      // H pieces, dH' pieces
      const int h = t / kGroups, g = t % kGroups;
      float v[8], w[8];
      wg_load8(sc_H, r0 + 8 * g, h, kHidden, n, v);
      wg_load8(sc_dH, r0 + 8 * g, h, kHidden, n, w);
      wg_store8(sm.Bh, nullptr, kmaj_off(h, 8 * g, kWgK), v);
      wg_store8(sm.Ad, nullptr, kmaj_off(h, 8 * g, kWgK), w);
      float v1[8], w1[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        v1[i] = __fsub_rn(v[i], __bfloat162float(__float2bfloat16_rn(v[i])));
        w1[i] = __fsub_rn(w[i], __bfloat162float(__float2bfloat16_rn(w[i])));
      }
      wg_store8(sm.Bh, nullptr, kmaj_off(kHidden + h, 8 * g, kWgK), v1);
      wg_store8(sm.Ad, nullptr, kmaj_off(kHidden + h, 8 * g, kWgK), w1);
    }
    for (int t = tid; t < in_dim * kGroups; t += kWgThreads) {       // X pieces
      const int i = t / kGroups, g = t % kGroups;
      float v[8], v1[8];
      wg_load8(sc_X, r0 + 8 * g, i, kMaxIn, n, v);
      wg_store8(sm.Bx, nullptr, kmaj_off(i, 8 * g, kWgK), v);
#pragma unroll
      for (int q = 0; q < 8; ++q) v1[q] = __fsub_rn(v[q], __bfloat162float(__float2bfloat16_rn(v[q])));
      wg_store8(sm.Bx, nullptr, kmaj_off(kMaxIn + i, 8 * g, kWgK), v1);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      constexpr uint32_t kId = make_idesc(128, kWgN);
      const uint32_t az0 = smem_u32(sm.Az[0]), az1 = smem_u32(sm.Az[1]), ad = smem_u32(sm.Ad);
      const uint32_t bh = smem_u32(sm.Bh), bx = smem_u32(sm.Bx);
#pragma unroll
      for (int kk = 0; kk < kWgK / 16; ++kk) {
        mma_bf16(tmem, kmaj_desc(az1, kWgK, 0, kk), kmaj_desc(bh, kWgK, 0, kk), kId, acc);
        mma_bf16(tmem, kmaj_desc(az0, kWgK, 0, kk), kmaj_desc(bh, kWgK, 0, kk), kId, 1u);
        mma_bf16(tmem + kWgW1Col, kmaj_desc(ad, kWgK, 0, kk), kmaj_desc(bx, kWgK, 0, kk), kId, acc);
        acc = 1;
      }
      mma_commit(mbar);
    }
    acc = 1;
    if (!__syncthreads_and(mbar_wait(mbar, phase))) { timed_out = true; break; }
    phase ^= 1u;
    fence_after();
  }
  // this CTA's sums -> its partial row (W2 row-major, b2, W1 row-major hidden x in_dim, b1)
  float* dst = partials + (long long)blockIdx.x * (kOut * kHidden + kOut + kHidden * in_dim + kHidden);
  const bool any = acc != 0 && !timed_out;
  if (warp < 4) {
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    const int m = warp * 32 + lane;
    float d[kWgN];
    {
      float a32[32], b32[32], c16[16];
      tmem_ld32(tl, a32);
      tmem_ld32(tl + 32, b32);
      tmem_ld16(tl + 64, c16);
#pragma unroll
      for (int i = 0; i < 32; ++i) { d[i] = a32[i]; d[32 + i] = b32[i]; }
#pragma unroll
      for (int i = 0; i < 16; ++i) d[64 + i] = c16[i];
    }
    if (m < kOut) {
      const bool colour = m >= kNOff && m < 4 * kNOff;
#pragma unroll
      for (int h = 0; h < kHidden; ++h) dst[m * kHidden + h] = any ? d[h] + (colour ? 0.f : d[kHidden + h]) : 0.f;
      dst[kOut * kHidden + m] = any ? d[2 * kHidden] : 0.f;
    }
    float e[kWgN];
    {
      float a32[32], b32[32], c16[16];
      tmem_ld32(tl + kWgW1Col, a32);
      tmem_ld32(tl + kWgW1Col + 32, b32);
      tmem_ld16(tl + kWgW1Col + 64, c16);
#pragma unroll
      for (int i = 0; i < 32; ++i) { e[i] = a32[i]; e[32 + i] = b32[i]; }
#pragma unroll
      for (int i = 0; i < 16; ++i) e[64 + i] = c16[i];
    }
    if (warp == 1) {
#pragma unroll
      for (int i = 0; i < kWgN; ++i) sm.red[lane][i] = e[i];
    }
    __syncwarp();
    if (warp < 2) asm volatile("bar.sync 1, 64;" ::: "memory");      // named barrier of warps 0 and 1 only
    if (warp == 0) {
      const int base = kOut * kHidden + kOut;
      for (int i = 0; i < in_dim; ++i)
        dst[base + lane * in_dim + i] = any ? e[i] + e[kMaxIn + i] + sm.red[lane][i] : 0.f;
      dst[base + kHidden * in_dim + lane] = any ? e[2 * kMaxIn] + sm.red[lane][2 * kMaxIn] : 0.f;
    }
  }
  if (timed_out) {
    if (tid == 0) set_flag(err, kFlagTimeout);
    (void)mbar_wait(mbar, phase);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kWgTmemCols);
  }
}

cudaError_t launch_mlp_wgrad_tc(const float* dZ, const float* H, const float* dH, const float* X,
                                const long long* n_rows, long long cap, int in_dim, float* partials, int nb_max,
                                const pgs_param_grad_ptrs& out, uint32_t* err, cudaStream_t st) {
  const size_t smem = sizeof(WgSmem) + 1024;
  prepare_smem_kernel(reinterpret_cast<const void*>(k_mlp_wgrad_tc), kWgThreads, smem);
  const long long chunks = (cap + kWgK - 1) / kWgK;
  const int nb = (int)std::max<long long>(1, std::min<long long>({chunks, (long long)device_sm_count(),
                                                                  (long long)nb_max}));
  k_mlp_wgrad_tc<<<nb, kWgThreads, smem, st>>>(dZ, H, dH, X, n_rows, cap, in_dim, partials, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_mlp_wgrad_final(partials, nb, in_dim, out, st);
}

cudaError_t launch_decode_bwd_tc(const BatchDev& b, const pgs_anchor_ptrs& A, const pgs_mlp_ptrs& W,
                                 const uint32_t* rows, const long long* n_rows, long long cap, const float* grad,
                                 const pgs_param_grad_ptrs& out, float* sc_dZ, float* sc_H, float* sc_dH, float* sc_X,
                                 uint32_t* err, cudaStream_t st) {
  const size_t smem = sizeof(BwdSmem) + 1024;
  const int per_sm = prepare_smem_kernel(reinterpret_cast<const void*>(k_decode_bwd_tc), kBwdThreads, smem);
  const long long tiles = (cap + kRows - 1) / kRows;
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)per_sm * device_sm_count()));
  k_decode_bwd_tc<<<grid, kBwdThreads, smem, st>>>(b, A, W, rows, n_rows, cap, grad, out, sc_dZ, sc_H, sc_dH, sc_X,
                                                   err);
  return cudaGetLastError();
}

}  // namespace pgs
