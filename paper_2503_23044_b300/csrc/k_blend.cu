// Front-to-back blending of RGB (Eq. 5), normal (Eq. 6) and plane distance
// with the unbiased depth D_hat = D / (N . K^-1 p~) (Eq. 7), and its reverse-
// order backward.
//
// One CTA per (view, tile) of the batch: two pixels per thread, the tile's
// sorted Gaussian list staged in shared memory in rounds of 256 records.
// The decisions of the forward (skip power > 0, skip alpha < alpha_min, clamp
// at alpha_max, stop before T drops below t_min) are taken with explicitly
// rounded operations so that the backward recomputes bit-identical alphas and
// walks exactly the forward's contributors, from the last one down, undoing
// the transmittance by division (T_i = T_{i+1} / (1 - alpha_i)).
#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

// scaled conic: power (log2 units) = A' dx^2 + C' dy^2 + B' dx dy
constexpr float kHalfLog2e = -0.5f * kLog2e;
constexpr float kNegLog2e = -kLog2e;
constexpr int kBatch = 256;   // records staged per round (two per thread)

struct BlendSmem {
  float4 m[kBatch];    // mean (hi x, hi y, lo x, lo y)
  float4 q[kBatch];    // (A', B', C', opacity)
  float4 c[kBatch];    // (r, g, b, d)
  float4 n[kBatch];    // (nx, ny, nz, p_lo): p_lo = log2(alpha_min / opacity)
};

// The alpha >= alpha_min rule is taken on the exponent, o 2^p >= alpha_min <=>
// p >= log2(alpha_min / o), so pairs below it never reach the exponential.
__device__ __forceinline__ void stage_record(BlendSmem& s, int slot, const float4* __restrict__ rec, uint32_t g,
                                             float a_min) {
  const float4* r = rec + (size_t)g * kRecF4;
  const float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3);
  s.m[slot] = r0;
  s.q[slot] = make_float4(__fmul_rn(r1.x, kHalfLog2e), __fmul_rn(r1.y, kNegLog2e), __fmul_rn(r1.z, kHalfLog2e), r1.w);
  s.c[slot] = r2;
  s.n[slot] = make_float4(r3.x, r3.y, r3.z, log2f(__fdiv_rn(a_min, r1.w)));
}

// power of the Gaussian at the pixel, with the exact operation order shared by both passes
__device__ __forceinline__ float eval_power(const float4 q, float dx, float dy) {
  return __fmaf_rn(q.x, __fmul_rn(dx, dx), __fmaf_rn(q.z, __fmul_rn(dy, dy), __fmul_rn(q.y, __fmul_rn(dx, dy))));
}
__device__ __forceinline__ float rel_d(float f_rel, float hi, float lo) { return __fsub_rn(__fsub_rn(f_rel, hi), lo); }

struct PixF {            // forward state of one pixel
  float fy, T, cr, cg, cb, D, n0, n1, n2;
  uint32_t last, ncontrib, stop;
  bool done;
};

__device__ __forceinline__ void fwd_pair(PixF& P, const BlendSmem& s, int k, uint32_t j, float dx, float4 q, float a_max,
                                         float t_min) {
  const float dy = rel_d(P.fy, s.m[k].y, s.m[k].w);
  const float power = eval_power(q, dx, dy);
  if (power > 0.f || !(power >= s.n[k].w)) return;
  const float a_raw = __fmul_rn(q.w, ex2_approx(power));
  const float alpha = fminf(a_max, a_raw);
  const float Tn = __fmul_rn(P.T, __fsub_rn(1.f, alpha));
  if (Tn < t_min) { P.done = true; P.stop = j + 1; return; }
  const float w = __fmul_rn(alpha, P.T);
  const float4 c = s.c[k], nn = s.n[k];
  P.cr = fmaf(w, c.x, P.cr); P.cg = fmaf(w, c.y, P.cg); P.cb = fmaf(w, c.z, P.cb); P.D = fmaf(w, c.w, P.D);
  P.n0 = fmaf(w, nn.x, P.n0); P.n1 = fmaf(w, nn.y, P.n1); P.n2 = fmaf(w, nn.z, P.n2);
  P.T = Tn;
  P.last = j + 1;
  ++P.ncontrib;
}

__device__ __forceinline__ void fwd_write(const PixF& P, const ViewDev& v, const ParamsDev& p, int px, int py,
                                          float fx_rel, uint32_t lo, const pgs_image_ptrs& out) {
  if (px >= v.W || py >= v.H) return;
  const long long HW = (long long)v.W * v.H;
  const long long q = v.pix_off + (long long)py * v.W + px;
  const long long q3 = 3 * v.pix_off + (long long)py * v.W + px;
  out.rgb[q3] = fmaf(P.T, p.bg, P.cr);
  out.rgb[q3 + HW] = fmaf(P.T, p.bg, P.cg);
  out.rgb[q3 + 2 * HW] = fmaf(P.T, p.bg, P.cb);
  out.normal[q3] = P.n0;
  out.normal[q3 + HW] = P.n1;
  out.normal[q3 + 2 * HW] = P.n2;
  // Eq. 7 with guards: |N . r| >= 1e-8 and accumulated weight >= 1e-6, else 0
  const float rx = fx_rel / v.fx, ry = P.fy / v.fy;
  const float ndr = P.n0 * rx + P.n1 * ry + P.n2;
  const bool ok = fabsf(ndr) >= 1e-8f && (1.f - P.T) >= 1e-6f;
  out.depth[q] = ok ? P.D / ndr : 0.f;
  out.dist[q] = P.D;
  out.t_final[q] = P.T;
  out.last[q] = P.last;
  if (out.n_contrib) out.n_contrib[q] = P.ncontrib;
  if (out.n_eval) out.n_eval[q] = P.stop - lo;
}

// Each thread owns two vertically adjacent pixels of the tile, so one staged
// record and its dx serve both; each warp covers a compact 8 x 8 block of the
// tile, so its pixels tend to agree on which Gaussians they skip or take.
template <int TW>
__device__ __forceinline__ void warp_block_pixel(int tx, int ty, int TH, int& px, int& py0) {
  const int w = (int)threadIdx.x >> 5, l = (int)threadIdx.x & 31;
  constexpr int WX = TW / 8;
  px = tx * TW + (w % WX) * 8 + (l & 7);
  py0 = ty * TH + (w / WX) * 8 + 2 * (l >> 3);
}
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2) k_blend_fwd(const __grid_constant__ BatchDev b,
                                                           const float4* __restrict__ rec,
                                                           const uint32_t* __restrict__ pair_g,
                                                           const uint2* __restrict__ ranges, pgs_image_ptrs out) {
  constexpr int NT = TW * TH / 2;
  static_assert(2 * NT == kBatch, "two records per thread per round");
  __shared__ BlendSmem s;
  const int tile = blockIdx.x;
  const int vi = view_of_tile(b, tile);
  const ViewDev& v = b.v[vi];
  const int lt = tile - v.tile_base;
  const int ty = lt / v.tiles_x, tx = lt - ty * v.tiles_x;
  int px, py0;
  warp_block_pixel<TW>(tx, ty, TH, px, py0);
  const float fx_rel = (float)px + 0.5f - v.cx;
  const uint2 rg = ranges[tile];
  const float a_min = b.p.alpha_min, a_max = b.p.alpha_max, t_min = b.p.t_min;
  PixF P0{(float)py0 + 0.5f - v.cy, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, rg.y, !(px < v.W && py0 < v.H)};
  PixF P1{(float)(py0 + 1) + 0.5f - v.cy, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, rg.y,
          !(px < v.W && py0 + 1 < v.H)};
  for (uint32_t start = rg.x; start < rg.y; start += kBatch) {
    if (__syncthreads_count(!(P0.done && P1.done)) == 0) break;
    const uint32_t j0 = start + threadIdx.x, j1 = j0 + NT;
    if (j0 < rg.y) stage_record(s, threadIdx.x, rec, pair_g[j0], a_min);
    if (j1 < rg.y) stage_record(s, threadIdx.x + NT, rec, pair_g[j1], a_min);
    __syncthreads();
    const int cnt = min((uint32_t)kBatch, rg.y - start);
    for (int k = 0; k < cnt; ++k) {
      if (P0.done && P1.done) break;
      const float4 q = s.q[k];
      const float dx = rel_d(fx_rel, s.m[k].x, s.m[k].z);
      const uint32_t j = start + k;
      if (!P0.done) fwd_pair(P0, s, k, j, dx, q, a_max, t_min);
      if (!P1.done) fwd_pair(P1, s, k, j, dx, q, a_max, t_min);
    }
  }
  fwd_write(P0, v, b.p, px, py0, fx_rel, rg.x, out);
  fwd_write(P1, v, b.p, px, py0 + 1, fx_rel, rg.x, out);
}

// Lane-distributed sum of 16 slots across a warp with 16 shuffles: afterwards
// lane l holds the warp total of slot (l >> 1) & 15.
__device__ __forceinline__ float warp_transpose_reduce16(float v[16], int lane) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool up = lane & 16;
    const float send = up ? v[i] : v[i + 8];
    const float keep = up ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool up = lane & 8;
    const float send = up ? v[i] : v[i + 4];
    const float keep = up ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool up = lane & 4;
    const float send = up ? v[i] : v[i + 2];
    const float keep = up ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool up = lane & 2;
    const float send = up ? v[0] : v[1];
    const float keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

struct PixB {            // backward state of one pixel
  float fy, T;
  float gC0, gC1, gC2, gD, gN0, gN1, gN2;       // dL/d(colour, D, N) at the pixel
  float GS;     // sum over channels of g_ch * (suffix sum of the later contributors' channel values)
  uint32_t last;
};

__device__ __forceinline__ void bwd_setup(PixB& P, const ViewDev& v, const ParamsDev& p, int px, int py, float fx_rel,
                                          const pgs_image_ptrs& img, const pgs_image_grad_ptrs& gi) {
  P.fy = (float)py + 0.5f - v.cy;
  P.T = 1.f; P.last = 0;
  P.gC0 = P.gC1 = P.gC2 = P.gD = P.gN0 = P.gN1 = P.gN2 = 0.f;
  P.GS = 0.f;
  if (px >= v.W || py >= v.H) return;
  const long long HW = (long long)v.W * v.H;
  const long long q = v.pix_off + (long long)py * v.W + px;
  const long long q3 = 3 * v.pix_off + (long long)py * v.W + px;
  P.last = img.last[q];
  P.T = img.t_final[q];
  P.gC0 = gi.rgb[q3]; P.gC1 = gi.rgb[q3 + HW]; P.gC2 = gi.rgb[q3 + 2 * HW];
  P.gN0 = gi.normal[q3]; P.gN1 = gi.normal[q3 + HW]; P.gN2 = gi.normal[q3 + 2 * HW];
  // chain through D_hat = D / (N . r)
  const float gDh = gi.depth[q];
  const float N0 = img.normal[q3], N1 = img.normal[q3 + HW], N2 = img.normal[q3 + 2 * HW];
  const float rx = fx_rel / v.fx, ry = P.fy / v.fy;
  const float ndr = N0 * rx + N1 * ry + N2;
  const bool ok = fabsf(ndr) >= 1e-8f && (1.f - P.T) >= 1e-6f;
  if (ok) {
    const float D = img.dist[q];
    const float ind = 1.f / ndr;
    P.gD = gDh * ind;
    const float k = -gDh * D * ind * ind;
    P.gN0 += k * rx; P.gN1 += k * ry; P.gN2 += k;
  }
  // the background enters the RGB suffix sums with weight T_final
  P.GS = P.T * p.bg * (P.gC0 + P.gC1 + P.gC2);
}

// Undo one contributor of the pixel (back to front) and add its per-pixel sums
// into vals; returns false if the pair did not contribute in the forward.
//   vals[0..5]  = sum G dx, G dy, G dx^2, G dx dy, G dy^2, G   (G = dL/dalpha * alpha_raw)
//   vals[6..12] = sum w gC (3), w gD, w gN (3)
// dL/dalpha_i = T_i (g . f_i) - (g . S_i) / (1 - alpha_i), with g . S_i carried as one scalar.
__device__ __forceinline__ bool bwd_pair(PixB& P, const BlendSmem& s, int k, float dx, float4 q, float a_max,
                                         float vals[16]) {
  const float dy = rel_d(P.fy, s.m[k].y, s.m[k].w);
  const float power = eval_power(q, dx, dy);
  const float4 nn = s.n[k];
  if (power > 0.f || !(power >= nn.w)) return false;
  const float a_raw = __fmul_rn(q.w, ex2_approx(power));
  const float alpha = fminf(a_max, a_raw);
  const float iom = 1.f / __fsub_rn(1.f, alpha);
  P.T = P.T * iom;
  const float w = alpha * P.T;
  const float4 c = s.c[k];
  float gf = P.gC0 * c.x;
  gf = fmaf(P.gC1, c.y, gf); gf = fmaf(P.gC2, c.z, gf); gf = fmaf(P.gD, c.w, gf);
  gf = fmaf(P.gN0, nn.x, gf); gf = fmaf(P.gN1, nn.y, gf); gf = fmaf(P.gN2, nn.z, gf);
  const float dLda = fmaf(P.T, gf, -P.GS * iom);
  P.GS = fmaf(w, gf, P.GS);
  vals[6] = fmaf(w, P.gC0, vals[6]); vals[7] = fmaf(w, P.gC1, vals[7]); vals[8] = fmaf(w, P.gC2, vals[8]);
  vals[9] = fmaf(w, P.gD, vals[9]);
  vals[10] = fmaf(w, P.gN0, vals[10]); vals[11] = fmaf(w, P.gN1, vals[11]); vals[12] = fmaf(w, P.gN2, vals[12]);
  if (!(a_raw > a_max)) {            // alpha clamped at alpha_max carries no gradient to o, mean, conic
    const float G = dLda * a_raw;
    vals[0] = fmaf(G, dx, vals[0]);
    vals[1] = fmaf(G, dy, vals[1]);
    vals[2] = fmaf(G, dx * dx, vals[2]);
    vals[3] = fmaf(G, dx * dy, vals[3]);
    vals[4] = fmaf(G, dy * dy, vals[4]);
    vals[5] += G;
  }
  return true;
}

// Per-Gaussian gradients from the reduced sums: power_nat = -1/2 (A dx^2 + 2B dx dy + C dy^2)
// with dx = px - mx, so d/dmx = A dx + B dy, d/dA = -1/2 dx^2, d/dB = -dx dy, d/dC = -1/2 dy^2,
// and d alpha / d o = alpha_raw / o.
__device__ __forceinline__ void finish_grads(const float* a, float4 q, float out[13]) {
  const float An = q.x * (1.f / kHalfLog2e), Bn = q.y * (1.f / kNegLog2e), Cn = q.z * (1.f / kHalfLog2e);
  out[0] = An * a[0] + Bn * a[1];
  out[1] = Bn * a[0] + Cn * a[1];
  out[2] = -0.5f * a[2];
  out[3] = -a[3];
  out[4] = -0.5f * a[4];
  out[5] = a[5] / q.w;
#pragma unroll
  for (int f = 6; f < 13; ++f) out[f] = a[f];
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2, 8) k_blend_bwd(const __grid_constant__ BatchDev b,
                                                           const float4* __restrict__ rec,
                                                           const uint32_t* __restrict__ pair_g,
                                                           const uint2* __restrict__ ranges, pgs_image_ptrs img,
                                                           pgs_image_grad_ptrs gi, float* __restrict__ grad) {
  constexpr int NT = TW * TH / 2;
  static_assert(2 * NT == kBatch, "two records per thread per round");
  __shared__ BlendSmem s;
  __shared__ float s_acc[kBatch][kGradFields];
  __shared__ uint32_t s_g[kBatch];
  __shared__ int s_max;
  const int tile = blockIdx.x;
  const uint2 rg = ranges[tile];
  if (rg.y <= rg.x) return;
  const int vi = view_of_tile(b, tile);
  const ViewDev& v = b.v[vi];
  const int lt = tile - v.tile_base;
  const int ty = lt / v.tiles_x, tx = lt - ty * v.tiles_x;
  int px, py0;
  warp_block_pixel<TW>(tx, ty, TH, px, py0);
  const float fx_rel = (float)px + 0.5f - v.cx;
  const int lane = threadIdx.x & 31;
  const float a_min = b.p.alpha_min, a_max = b.p.alpha_max;
  PixB P0, P1;
  bwd_setup(P0, v, b.p, px, py0, fx_rel, img, gi);
  bwd_setup(P1, v, b.p, px, py0 + 1, fx_rel, img, gi);
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  atomicMax(&s_max, (int)max(P0.last, P1.last));
  __syncthreads();
  const uint32_t end = (uint32_t)s_max;   // 1 + last contributor index over the tile
  for (uint32_t bend = end; bend > rg.x;) {
    const uint32_t bstart = bend > rg.x + kBatch ? bend - kBatch : rg.x;
    const int cnt = (int)(bend - bstart);
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int slot = threadIdx.x + h * NT;
      if (slot < cnt) {
        const uint32_t g = pair_g[bstart + slot];
        s_g[slot] = g;
        stage_record(s, slot, rec, g, a_min);
#pragma unroll
        for (int f = 0; f < kGradFields; ++f) s_acc[slot][f] = 0.f;
      }
    }
    __syncthreads();
    // the warp walks from its highest live index down
    const int my_top = (int)min(max(P0.last, P1.last), bend) - 1 - (int)bstart;
    const int top = __reduce_max_sync(0xffffffffu, my_top);
    for (int k = top; k >= 0; --k) {
      const uint32_t j = bstart + k;
      float vals[16];
#pragma unroll
      for (int f = 0; f < 16; ++f) vals[f] = 0.f;
      bool contrib = false;
      const bool live0 = j < P0.last, live1 = j < P1.last;
      if (live0 || live1) {
        const float4 q = s.q[k];
        const float dx = rel_d(fx_rel, s.m[k].x, s.m[k].z);
        if (live0) contrib |= bwd_pair(P0, s, k, dx, q, a_max, vals);
        if (live1) contrib |= bwd_pair(P1, s, k, dx, q, a_max, vals);
      }
      if (__any_sync(0xffffffffu, contrib)) {
        const float r = warp_transpose_reduce16(vals, lane);
        const int slot = (lane >> 1) & 15;
        if (!(lane & 1) && slot < kGradFields) atomicAdd(&s_acc[k][slot], r);
      }
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int slot = threadIdx.x + h * NT;
      if (slot < cnt) {
        float a[13];
        finish_grads(s_acc[slot], s.q[slot], a);
        float4* dst = reinterpret_cast<float4*>(grad + (size_t)s_g[slot] * 16);
        const float4 v0 = make_float4(a[0], a[1], a[2], a[3]);
        const float4 v1 = make_float4(a[4], a[5], a[6], a[7]);
        const float4 v2 = make_float4(a[8], a[9], a[10], a[11]);
        if (v0.x != 0.f || v0.y != 0.f || v0.z != 0.f || v0.w != 0.f) atomicAdd(dst, v0);
        if (v1.x != 0.f || v1.y != 0.f || v1.z != 0.f || v1.w != 0.f) atomicAdd(dst + 1, v1);
        if (v2.x != 0.f || v2.y != 0.f || v2.z != 0.f || v2.w != 0.f) atomicAdd(dst + 2, v2);
        if (a[12] != 0.f) atomicAdd(reinterpret_cast<float*>(dst + 3), a[12]);
      }
    }
    bend = bstart;
  }
}

template <int TW, int TH>
static void launch_fwd_t(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                         const pgs_image_ptrs& o, cudaStream_t st) {
  k_blend_fwd<TW, TH><<<b.total_tiles, TW * TH / 2, 0, st>>>(b, rec, pg, rg, o);
}
template <int TW, int TH>
static void launch_bwd_t(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                         const pgs_image_ptrs& img, const pgs_image_grad_ptrs& gi, float* grad, cudaStream_t st) {
  k_blend_bwd<TW, TH><<<b.total_tiles, TW * TH / 2, 0, st>>>(b, rec, pg, rg, img, gi, grad);
}

bool launch_blend_fwd(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                      const pgs_image_ptrs& o, cudaStream_t st) {
  const int tw = b.p.tile_w, th = b.p.tile_h;
  if (tw == 16 && th == 16) launch_fwd_t<16, 16>(b, rec, pg, rg, o, st);
  else if (tw == 8 && th == 32) launch_fwd_t<8, 32>(b, rec, pg, rg, o, st);
  else if (tw == 32 && th == 8) launch_fwd_t<32, 8>(b, rec, pg, rg, o, st);
  else return false;
  return true;
}

bool launch_blend_bwd(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                      const pgs_image_ptrs& img, const pgs_image_grad_ptrs& gi, float* grad, cudaStream_t st) {
  const int tw = b.p.tile_w, th = b.p.tile_h;
  if (tw == 16 && th == 16) launch_bwd_t<16, 16>(b, rec, pg, rg, img, gi, grad, st);
  else if (tw == 8 && th == 32) launch_bwd_t<8, 32>(b, rec, pg, rg, img, gi, grad, st);
  else if (tw == 32 && th == 8) launch_bwd_t<32, 8>(b, rec, pg, rg, img, gi, grad, st);
  else return false;
  return true;
}

}  // namespace pgs
