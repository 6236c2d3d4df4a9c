// Backward of the EWA projection and of the shared decoder (Eq. 4).
//
// Per Gaussian-view the blend backward left 13 gradients (2D mean, conic,
// opacity, colour, plane distance d, normal).  Here they are chained through
// the projection (conic -> 2D covariance -> J and Sigma -> scale and rotation;
// 2D mean -> camera-frame mean; normal and d -> rotation and mean; the normal's
// axis choice and facing sign are held fixed) and, in anchor mode, through the
// decoder's activations and both linear layers.  Per-anchor gradients are
// summed over the views of the batch with atomics; the decoder's weight
// gradients, summed over all visible (view, anchor) rows, go through a
// split-row reduction with fixed-order partial sums.
#include <cuda_bf16.h>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"
#include "pgs_backward.cuh"

namespace pgs {

// ---------------------------------------------------------------- explicit mode
__global__ void __launch_bounds__(128) k_project_bwd_explicit(const __grid_constant__ BatchDev b, pgs_explicit_ptrs P,
                                                              long long N, const float* __restrict__ grad,
                                                              pgs_param_grad_ptrs out, uint32_t* err) {
  const long long G = N * b.n_views;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
    float gr[13];
    if (!load_grad(grad, g, gr)) continue;
    const int vi = (int)(g / N);
    const long long i = g - (long long)vi * N;
    const float mu[3] = {P.means[3 * i], P.means[3 * i + 1], P.means[3 * i + 2]};
    const float s[3] = {expf(P.log_scales[3 * i]), expf(P.log_scales[3 * i + 1]), expf(P.log_scales[3 * i + 2])};
    const float qr[4] = {P.quats[4 * i], P.quats[4 * i + 1], P.quats[4 * i + 2], P.quats[4 * i + 3]};
    const float qn = sqrtf(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    float q[4] = {1.f, 0.f, 0.f, 0.f};
    if (qn >= 1e-12f) { const float iq = 1.f / qn; for (int t = 0; t < 4; ++t) q[t] = qr[t] * iq; }
    ProjGrad pg;
    project_backward(b, b.v[vi], mu, s, q, gr, pg);
    float dq[4];
    quat_norm_backward(qr, qn, pg.dq, dq);
    const float op = sigm(P.opacity_logits[i]);
    bool bad = false;
    for (int t = 0; t < 3; ++t) {
      add_if(out.means ? out.means + 3 * i + t : nullptr, pg.dmu[t]);
      add_if(out.log_scales ? out.log_scales + 3 * i + t : nullptr, pg.ds[t] * s[t]);
      add_if(out.colors ? out.colors + 3 * i + t : nullptr, pg.dcol[t]);
      bad |= !isfinite(pg.dmu[t]) || !isfinite(pg.ds[t]);
    }
    for (int t = 0; t < 4; ++t) add_if(out.quats ? out.quats + 4 * i + t : nullptr, dq[t]);
    add_if(out.opacity_logits ? out.opacity_logits + i : nullptr, pg.dop * op * (1.f - op));
    if (bad) set_flag(err, kFlagNonfinite);
  }
}

// ---------------------------------------------------------------- anchor mode
struct __align__(16) MlpSmemB {
  float W1[kHidden][kMaxIn];   // zero past in_dim; rows are 16-byte aligned (36 floats)
  float b1[kHidden];
  float W2[kOut][kHidden];     // rows of 32 floats
  float b2[kOut];
};
static_assert(kMaxIn % 4 == 0 && kHidden % 4 == 0, "float4 rows");

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ bool colour_out(int o) { return o >= kNOff && o < 4 * kNOff; }

// z = b2[o] + W2[o] . H (one decoder output, weight row read as float4); with
// round_h the hidden values are rounded to BF16 first (the one-pass colour
// heads of the BF16 decoder, whose weight rows are stored rounded)
__device__ __forceinline__ float w2_dot(const MlpSmemB& m, int o, const float (&H)[kHidden], bool round_h) {
  const float4* w = reinterpret_cast<const float4*>(m.W2[o]);
  float acc = m.b2[o];
  if (round_h) {
#pragma unroll
    for (int q = 0; q < kHidden / 4; ++q) {
      const float4 ww = w[q];
      acc = fmaf(ww.x, bf16r(H[4 * q]), acc); acc = fmaf(ww.y, bf16r(H[4 * q + 1]), acc);
      acc = fmaf(ww.z, bf16r(H[4 * q + 2]), acc); acc = fmaf(ww.w, bf16r(H[4 * q + 3]), acc);
    }
    return acc;
  }
#pragma unroll
  for (int q = 0; q < kHidden / 4; ++q) {
    const float4 ww = w[q];
    acc = fmaf(ww.x, H[4 * q], acc); acc = fmaf(ww.y, H[4 * q + 1], acc);
    acc = fmaf(ww.z, H[4 * q + 2], acc); acc = fmaf(ww.w, H[4 * q + 3], acc);
  }
  return acc;
}
// dH += W2[o]^T dz (one decoder output's contribution to the hidden-layer gradient)
__device__ __forceinline__ void w2_axpy(const MlpSmemB& m, int o, float dz, float (&dH)[kHidden]) {
  const float4* w = reinterpret_cast<const float4*>(m.W2[o]);
#pragma unroll
  for (int q = 0; q < kHidden / 4; ++q) {
    const float4 ww = w[q];
    dH[4 * q] = fmaf(ww.x, dz, dH[4 * q]); dH[4 * q + 1] = fmaf(ww.y, dz, dH[4 * q + 1]);
    dH[4 * q + 2] = fmaf(ww.z, dz, dH[4 * q + 2]); dH[4 * q + 3] = fmaf(ww.w, dz, dH[4 * q + 3]);
  }
}

// Per visible row: recompute the decoder forward (H, then each Gaussian's 11
// outputs), run the projection backward of its 10 Gaussians, and carry the
// gradient back through the decoder: dZ (11 entries per Gaussian, written to
// the weight-gradient scratch as they are formed), dH accumulated in registers
// Gaussian by Gaussian, dX = W1^T (dH . [H > 0]).  The recomputed forward
// rounds where the rendered one did (b.p.decode): the BF16 decoder's colour
// heads multiply BF16-rounded H and W2 rows; the one-pass form rounds X, W1,
// H and W2.  The gradient passes straight through each rounding, i.e. the
// backward multiplies the same rounded operands the forward multiplied.
__global__ void __launch_bounds__(128) k_decode_bwd(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A,
                                                    pgs_mlp_ptrs Wt, const uint32_t* __restrict__ rows,
                                                    const long long* __restrict__ n_rows_p, long long cap,
                                                    const float* __restrict__ grad, pgs_param_grad_ptrs out,
                                                    float* __restrict__ sc_dZ, float* __restrict__ sc_H,
                                                    float* __restrict__ sc_dH, float* __restrict__ sc_X, uint32_t* err) {
  __shared__ MlpSmemB m;
  const int in_dim = b.p.in_dim;
  const bool one_pass = b.p.decode == PGS_DECODE_BF16_1PASS;
  const bool round_colour = b.p.decode == PGS_DECODE_BF16;
  for (int t = threadIdx.x; t < kHidden * kMaxIn; t += blockDim.x) {
    const int i = t / kMaxIn, j = t % kMaxIn;
    const float w = j < in_dim ? Wt.W1[i * in_dim + j] : 0.f;
    m.W1[i][j] = one_pass ? bf16r(w) : w;
  }
  for (int t = threadIdx.x; t < kHidden; t += blockDim.x) m.b1[t] = Wt.b1[t];
  for (int t = threadIdx.x; t < kOut * kHidden; t += blockDim.x) {
    const float w = Wt.W2[t];
    m.W2[t / kHidden][t % kHidden] = (one_pass || (round_colour && colour_out(t / kHidden))) ? bf16r(w) : w;
  }
  for (int t = threadIdx.x; t < kOut; t += blockDim.x) m.b2[t] = Wt.b2[t];
  __syncthreads();
  const long long n_rows = min(*n_rows_p, cap);
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n_rows;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t rw = rows[r];
    const int vi = rw >> 27;
    const long long a = rw & ((1u << 27) - 1);
    const ViewDev& v = b.v[vi];
    float H[kHidden];
    float dir0, dir1, dir2, idist;
    {
      float X[kMaxIn];
      const float ddx = A.x[3 * a] - v.center[0], ddy = A.x[3 * a + 1] - v.center[1], ddz = A.x[3 * a + 2] - v.center[2];
      const float dist = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
      idist = 1.f / dist;
#pragma unroll
      for (int j = 0; j < kFeat; ++j) X[j] = A.feat[a * kFeat + j];
      dir0 = ddx * idist; dir1 = ddy * idist; dir2 = ddz * idist;
      X[32] = dir0; X[33] = dir1; X[34] = dir2;
      X[35] = in_dim == 36 ? dist : 0.f;
      if (one_pass) {
#pragma unroll
        for (int j = 0; j < kMaxIn; ++j) X[j] = bf16r(X[j]);
      }
#pragma unroll
      for (int i = 0; i < kHidden; ++i) {
        const float4* w = reinterpret_cast<const float4*>(m.W1[i]);
        float acc = m.b1[i];
#pragma unroll
        for (int q = 0; q < kMaxIn / 4; ++q) {
          const float4 ww = w[q];
          acc = fmaf(ww.x, X[4 * q], acc); acc = fmaf(ww.y, X[4 * q + 1], acc);
          acc = fmaf(ww.z, X[4 * q + 2], acc); acc = fmaf(ww.w, X[4 * q + 3], acc);
        }
        H[i] = one_pass ? bf16r(fmaxf(acc, 0.f)) : fmaxf(acc, 0.f);
      }
      // row scratch for the weight gradients, in 32-row blocks (sc_at)
#pragma unroll
      for (int j = 0; j < kMaxIn; ++j)
        if (j < in_dim) sc_X[sc_at(r, j, kMaxIn)] = X[j];
    }
#pragma unroll
    for (int h = 0; h < kHidden; ++h) sc_H[sc_at(r, h, kHidden)] = H[h];
    const float l[3] = {expf(A.log_l[3 * a]), expf(A.log_l[3 * a + 1]), expf(A.log_l[3 * a + 2])};
    const float xa[3] = {A.x[3 * a], A.x[3 * a + 1], A.x[3 * a + 2]};
    float dH[kHidden];
#pragma unroll
    for (int h = 0; h < kHidden; ++h) dH[h] = 0.f;
    float dl[3] = {0.f, 0.f, 0.f}, dxa[3] = {0.f, 0.f, 0.f};
    bool any = false, bad = false;
#pragma unroll 1
    for (int j = 0; j < kNOff; ++j) {
      const int idx[11] = {j, 10 + 3 * j, 11 + 3 * j, 12 + 3 * j, 40 + 3 * j, 41 + 3 * j, 42 + 3 * j,
                           70 + 4 * j, 71 + 4 * j, 72 + 4 * j, 73 + 4 * j};
      float dz[11];
      float gr[13];
      if (!load_grad(grad, r * kNOff + j, gr)) {
#pragma unroll
        for (int t = 0; t < 11; ++t) sc_dZ[sc_at(r, idx[t], kOut)] = 0.f;
        continue;
      }
      any = true;
      float z[11];
#pragma unroll
      for (int t = 0; t < 11; ++t) z[t] = w2_dot(m, idx[t], H, round_colour && t >= 1 && t <= 3);
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
      project_backward(b, v, mu, s, q, gr, pg);
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
#pragma unroll
      for (int t = 0; t < 11; ++t) {
        sc_dZ[sc_at(r, idx[t], kOut)] = dz[t];
        w2_axpy(m, idx[t], dz[t], dH);
      }
    }
    // hidden layer: dH_pre = (W2^T dZ) * [H > 0]
#pragma unroll
    for (int h = 0; h < kHidden; ++h) {
      dH[h] = H[h] > 0.f ? dH[h] : 0.f;
      sc_dH[sc_at(r, h, kHidden)] = dH[h];
    }
    if (any) {
      // input: dX = W1^T dH_pre (feature part to out.feat, direction part to the anchor position)
      float dX[kMaxIn];
#pragma unroll
      for (int j = 0; j < kMaxIn; ++j) dX[j] = 0.f;
#pragma unroll
      for (int i = 0; i < kHidden; ++i) {
        const float4* w = reinterpret_cast<const float4*>(m.W1[i]);
#pragma unroll
        for (int qd = 0; qd < kMaxIn / 4; ++qd) {
          const float4 ww = w[qd];
          dX[4 * qd] = fmaf(ww.x, dH[i], dX[4 * qd]); dX[4 * qd + 1] = fmaf(ww.y, dH[i], dX[4 * qd + 1]);
          dX[4 * qd + 2] = fmaf(ww.z, dH[i], dX[4 * qd + 2]); dX[4 * qd + 3] = fmaf(ww.w, dH[i], dX[4 * qd + 3]);
        }
      }
#pragma unroll
      for (int j = 0; j < kFeat; ++j) add_if(out.feat ? out.feat + a * kFeat + j : nullptr, dX[j]);
      // unit view direction dir = (x - o)/|x - o|: d dir / dx = (I - dir dir^T) / |x - o|
      const float dd = dir0 * dX[32] + dir1 * dX[33] + dir2 * dX[34];
      dxa[0] += (dX[32] - dir0 * dd) * idist;
      dxa[1] += (dX[33] - dir1 * dd) * idist;
      dxa[2] += (dX[34] - dir2 * dd) * idist;
      if (in_dim == 36) { dxa[0] += dX[35] * dir0; dxa[1] += dX[35] * dir1; dxa[2] += dX[35] * dir2; }
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        add_if(out.x ? out.x + 3 * a + t : nullptr, dxa[t]);
        add_if(out.log_l ? out.log_l + 3 * a + t : nullptr, dl[t] * l[t]);
      }
    }
    if (bad) set_flag(err, kFlagNonfinite);
  }
}

// ---------------------------------------------------------------- decoder weight gradients
// dW2 = sum_r dZ_r H_r^T, db2 = sum_r dZ_r, dW1 = sum_r dH_r X_r^T, db1 = sum_r dH_r.
// Block b reduces a fixed contiguous slice of rows into partials[b][.]; a second
// kernel adds the partials in block order (deterministic) into the outputs.
constexpr int kWgRows = 32;

__host__ __device__ inline int wgrad_outputs(int in_dim) { return kOut * kHidden + kOut + kHidden * in_dim + kHidden; }

// Each block stages kWgRows rows at a time row-major in shared memory and
// accumulates register tiles.  Warps 0..5 hold 5 x 4 tiles of dW2 (110 x 32; 176
// of their 192 threads), warps 6..7 hold 4 x 5 tiles of dW1 (32 x in_dim); a
// thread whose tile starts at column 0 also sums its rows of dZ (db2) or dH
// (db1).  Every warp runs one code path, and the next round's scratch is loaded
// into registers while the current round is summed.
constexpr int kWgZ = kOut + 1, kWgH = kHidden + 1, kWgX = kMaxIn + 1;   // padded row strides
constexpr int kWgTilesW2 = (kOut / 5) * (kHidden / 4);                   // 176
constexpr int kWgTilesW1 = (kHidden / 4) * ((kMaxIn + 4) / 5);           // 64
constexpr int kWgRole1 = 192;                                            // first dW1 thread (warp 6)
static_assert(kOut % 5 == 0 && kHidden % 4 == 0, "tile shapes");
static_assert(kWgTilesW2 <= kWgRole1 && kWgRole1 + kWgTilesW1 == 256, "thread roles");

struct WgStage {
  static constexpr int kNZ = (kOut * kWgRows + 255) / 256, kNH = kHidden * kWgRows / 256;
  static constexpr int kNX = (kMaxIn * kWgRows + 255) / 256;
  float z[kNZ], h[kNH], dh[kNH], x[kNX];
};

// load one 32-row scratch block (rows rb .. rb + nr - 1) into registers: thread t
// takes row t % 32 of features t / 32 + 8 k
__device__ __forceinline__ void wg_load(WgStage& v, const float* __restrict__ sc_dZ, const float* __restrict__ sc_H,
                                        const float* __restrict__ sc_dH, const float* __restrict__ sc_X, long long rb,
                                        int nr, int in_dim) {
  const int t = threadIdx.x, rr = t % kWgRows, i0 = t / kWgRows;
  const bool rok = rr < nr;
#pragma unroll
  for (int k = 0; k < WgStage::kNZ; ++k) {
    const int i = i0 + 8 * k;
    v.z[k] = (rok && i < kOut) ? sc_dZ[sc_at(rb + rr, i, kOut)] : 0.f;
  }
#pragma unroll
  for (int k = 0; k < WgStage::kNH; ++k) {
    const int i = i0 + 8 * k;
    v.h[k] = rok ? sc_H[sc_at(rb + rr, i, kHidden)] : 0.f;
    v.dh[k] = rok ? sc_dH[sc_at(rb + rr, i, kHidden)] : 0.f;
  }
#pragma unroll
  for (int k = 0; k < WgStage::kNX; ++k) {
    const int i = i0 + 8 * k;
    v.x[k] = (rok && i < in_dim) ? sc_X[sc_at(rb + rr, i, kMaxIn)] : 0.f;
  }
}

// launched with exactly 256 threads (the staging assumes it)
__global__ void __launch_bounds__(256) k_mlp_wgrad_partial(const float* __restrict__ sc_dZ, const float* __restrict__ sc_H,
                                                           const float* __restrict__ sc_dH, const float* __restrict__ sc_X,
                                                           const long long* __restrict__ n_rows_p, long long cap,
                                                           int in_dim, int round_colour_h,
                                                           float* __restrict__ partials) {
  __shared__ float sZ[kWgRows][kWgZ];
  __shared__ float sH[kWgRows][kWgH];
  __shared__ float sdH[kWgRows][kWgH];
  __shared__ float sX[kWgRows][kWgX];
  const long long n = min(*n_rows_p, cap);
  // whole 32-row scratch blocks per CTA, so each round reads one contiguous block per array
  const long long per = ((n + gridDim.x - 1) / gridDim.x + kScBlock - 1) / kScBlock * kScBlock;
  const long long r0 = min(n, (long long)blockIdx.x * per), r1 = min(n, r0 + per);
  const int n_out = wgrad_outputs(in_dim);
  const int t = threadIdx.x;
  const bool w2 = t < kWgRole1;
  const bool live = w2 ? t < kWgTilesW2 : true;
  int fa, gb;
  if (w2) { fa = (min(t, kWgTilesW2 - 1) / (kHidden / 4)) * 5; gb = (min(t, kWgTilesW2 - 1) % (kHidden / 4)) * 4; }
  else { const int u = t - kWgRole1; fa = (u / ((kMaxIn + 4) / 5)) * 4; gb = (u % ((kMaxIn + 4) / 5)) * 5; }
  const bool bias = gb == 0;          // also sums the bias entries of its rows
  // dW2 tiles of colour outputs (rows 10..39, whole 5-row tiles) multiply BF16-rounded H in the BF16 form
  const bool round_h = w2 && round_colour_h && fa >= kNOff && fa < 4 * kNOff;
  float acc[20], bs[5];
#pragma unroll
  for (int i = 0; i < 20; ++i) acc[i] = 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) bs[i] = 0.f;
  const int rr_s = t % kWgRows, i0_s = t / kWgRows;
  WgStage v;
  if (r0 < r1) wg_load(v, sc_dZ, sc_H, sc_dH, sc_X, r0, (int)min((long long)kWgRows, r1 - r0), in_dim);
  for (long long rb = r0; rb < r1; rb += kWgRows) {
    __syncthreads();                  // the previous round's tiles are consumed
#pragma unroll
    for (int k = 0; k < WgStage::kNZ; ++k)
      if (i0_s + 8 * k < kOut) sZ[rr_s][i0_s + 8 * k] = v.z[k];
#pragma unroll
    for (int k = 0; k < WgStage::kNH; ++k) { sH[rr_s][i0_s + 8 * k] = v.h[k]; sdH[rr_s][i0_s + 8 * k] = v.dh[k]; }
#pragma unroll
    for (int k = 0; k < WgStage::kNX; ++k)
      if (i0_s + 8 * k < kMaxIn) sX[rr_s][i0_s + 8 * k] = v.x[k];
    __syncthreads();
    const long long nb2 = rb + kWgRows;
    if (nb2 < r1) wg_load(v, sc_dZ, sc_H, sc_dH, sc_X, nb2, (int)min((long long)kWgRows, r1 - nb2), in_dim);
    if (w2) {
#pragma unroll 4
      for (int rr = 0; rr < kWgRows; ++rr) {
        float u[5], w[4];
#pragma unroll
        for (int a = 0; a < 5; ++a) u[a] = sZ[rr][fa + a];
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = round_h ? bf16r(sH[rr][gb + c]) : sH[rr][gb + c];
#pragma unroll
        for (int a = 0; a < 5; ++a) {
          bs[a] += u[a];
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a * 4 + c] = fmaf(u[a], w[c], acc[a * 4 + c]);
        }
      }
    } else {
#pragma unroll 4
      for (int rr = 0; rr < kWgRows; ++rr) {
        float u[4], w[5];
#pragma unroll
        for (int a = 0; a < 4; ++a) u[a] = sdH[rr][fa + a];
#pragma unroll
        for (int c = 0; c < 5; ++c) w[c] = sX[rr][min(gb + c, kMaxIn - 1)];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          bs[a] += u[a];
#pragma unroll
          for (int c = 0; c < 5; ++c) acc[a * 5 + c] = fmaf(u[a], w[c], acc[a * 5 + c]);
        }
      }
    }
  }
  // outputs in the order W2 (row-major), b2, W1 (row-major, hidden x in_dim), b1
  float* dst = partials + (long long)blockIdx.x * n_out;
  if (w2 && live) {
#pragma unroll
    for (int a = 0; a < 5; ++a) {
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[(fa + a) * kHidden + gb + c] = acc[a * 4 + c];
      if (bias) dst[kOut * kHidden + fa + a] = bs[a];
    }
  } else if (!w2) {
    const int base = kOut * kHidden + kOut;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int c = 0; c < 5; ++c)
        if (gb + c < in_dim) dst[base + (fa + a) * in_dim + gb + c] = acc[a * 5 + c];
      if (bias) dst[base + kHidden * in_dim + fa + a] = bs[a];
    }
  }
}

// Sum of the per-block partials in block order: warp w of a block adds blocks
// w, w + 8, ... for 32 consecutive outputs, then the 8 warp sums are added in
// warp order (fixed order, so the result is reproducible).
__global__ void __launch_bounds__(256) k_mlp_wgrad_final(const float* __restrict__ partials, int nb, int in_dim,
                                                         pgs_param_grad_ptrs out) {
  __shared__ float s_part[8][32];
  const int n_out = wgrad_outputs(in_dim);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (o < n_out) {
    int k = w;
    for (; k + 56 < nb; k += 64) {     // eight independent loads per round, added in block order
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = partials[(long long)(k + 8 * u) * n_out + o];
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; k < nb; k += 8) s += partials[(long long)k * n_out + o];
  }
  s_part[w][lane] = s;
  __syncthreads();
  if (w != 0 || o >= n_out) return;
  float tot = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) tot += s_part[k][lane];
  float* dst;
  if (o < kOut * kHidden) dst = out.W2 ? out.W2 + o : nullptr;
  else if (o < kOut * kHidden + kOut) dst = out.b2 ? out.b2 + (o - kOut * kHidden) : nullptr;
  else if (o < kOut * kHidden + kOut + kHidden * in_dim) dst = out.W1 ? out.W1 + (o - kOut * kHidden - kOut) : nullptr;
  else dst = out.b1 ? out.b1 + (o - kOut * kHidden - kOut - kHidden * in_dim) : nullptr;
  if (dst) *dst += tot;
}

int mlp_wgrad_outputs(int in_dim) { return wgrad_outputs(in_dim); }

cudaError_t launch_mlp_wgrad_final(const float* partials, int nb, int in_dim, const pgs_param_grad_ptrs& out,
                                   cudaStream_t st) {
  k_mlp_wgrad_final<<<(wgrad_outputs(in_dim) + 31) / 32, 256, 0, st>>>(partials, nb, in_dim, out);
  return cudaGetLastError();
}

void launch_mlp_wgrad(const float* dZ, const float* H, const float* dH, const float* X, const long long* n_rows,
                      long long cap, int in_dim, bool round_colour_h, float* partials, int nb,
                      const pgs_param_grad_ptrs& out, cudaStream_t st) {
  k_mlp_wgrad_partial<<<nb, 256, 0, st>>>(dZ, H, dH, X, n_rows, cap, in_dim, round_colour_h ? 1 : 0, partials);
  k_mlp_wgrad_final<<<(wgrad_outputs(in_dim) + 31) / 32, 256, 0, st>>>(partials, nb, in_dim, out);
}

}  // namespace pgs
