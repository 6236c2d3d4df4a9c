// Front-to-back blending of RGB (Eq. 5), normal (Eq. 6) and plane distance
// with the unbiased depth D_hat = D / (N . K^-1 p~) (Eq. 7), and its reverse-
// order backward.
//
// One CTA per (view, tile) of the batch: one thread per pixel, the tile's
// sorted Gaussian list staged in shared memory in batches of TW*TH records.
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

struct BlendSmem {
  float4 m[256];    // mean (hi x, hi y, lo x, lo y)
  float4 q[256];    // (A', B', C', opacity)
  float4 c[256];    // (r, g, b, d)
  float4 n[256];    // (nx, ny, nz, unused)
};

__device__ __forceinline__ void stage_record(BlendSmem& s, int slot, const float4* __restrict__ rec, uint32_t g) {
  const float4* r = rec + (size_t)g * kRecF4;
  const float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3);
  s.m[slot] = r0;
  s.q[slot] = make_float4(__fmul_rn(r1.x, kHalfLog2e), __fmul_rn(r1.y, kNegLog2e), __fmul_rn(r1.z, kHalfLog2e), r1.w);
  s.c[slot] = r2;
  s.n[slot] = r3;
}

// power of the Gaussian at the pixel, with the exact operation order shared by both passes
__device__ __forceinline__ float eval_power(const float4 m, const float4 q, float fx_rel, float fy_rel, float& dx,
                                            float& dy) {
  dx = __fsub_rn(__fsub_rn(fx_rel, m.x), m.z);
  dy = __fsub_rn(__fsub_rn(fy_rel, m.y), m.w);
  return __fmaf_rn(q.x, __fmul_rn(dx, dx), __fmaf_rn(q.z, __fmul_rn(dy, dy), __fmul_rn(q.y, __fmul_rn(dx, dy))));
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) k_blend_fwd(const __grid_constant__ BatchDev b,
                                                       const float4* __restrict__ rec,
                                                       const uint32_t* __restrict__ pair_g,
                                                       const uint2* __restrict__ ranges, pgs_image_ptrs out) {
  constexpr int NT = TW * TH;
  __shared__ BlendSmem s;
  const int tile = blockIdx.x;
  const int vi = view_of_tile(b, tile);
  const ViewDev& v = b.v[vi];
  const int lt = tile - v.tile_base;
  const int ty = lt / v.tiles_x, tx = lt - ty * v.tiles_x;
  const int px = tx * TW + (int)threadIdx.x % TW, py = ty * TH + (int)threadIdx.x / TW;
  const bool inside = px < v.W && py < v.H;
  const float fx_rel = (float)px + 0.5f - v.cx, fy_rel = (float)py + 0.5f - v.cy;
  const uint2 rg = ranges[tile];
  const float a_min = b.p.alpha_min, a_max = b.p.alpha_max, t_min = b.p.t_min;
  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, D = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
  uint32_t last = 0, ncontrib = 0, neval = 0;
  bool done = !inside;
  for (uint32_t start = rg.x; start < rg.y; start += NT) {
    if (__syncthreads_count(!done) == 0) break;
    const uint32_t j = start + threadIdx.x;
    if (j < rg.y) stage_record(s, threadIdx.x, rec, pair_g[j]);
    __syncthreads();
    if (!done) {
      const int cnt = min((uint32_t)NT, rg.y - start);
      for (int k = 0; k < cnt; ++k) {
        float dx, dy;
        const float power = eval_power(s.m[k], s.q[k], fx_rel, fy_rel, dx, dy);
        ++neval;
        if (power > 0.f) continue;
        const float a_raw = __fmul_rn(s.q[k].w, ex2_approx(power));
        if (a_raw < a_min) continue;
        const float alpha = fminf(a_max, a_raw);
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
        if (Tn < t_min) { done = true; break; }
        const float w = __fmul_rn(alpha, T);
        const float4 c = s.c[k], nn = s.n[k];
        cr = fmaf(w, c.x, cr); cg = fmaf(w, c.y, cg); cb = fmaf(w, c.z, cb); D = fmaf(w, c.w, D);
        n0 = fmaf(w, nn.x, n0); n1 = fmaf(w, nn.y, n1); n2 = fmaf(w, nn.z, n2);
        T = Tn;
        last = start + k + 1;
        ++ncontrib;
      }
    }
  }
  if (!inside) return;
  const long long HW = (long long)v.W * v.H;
  const long long p = v.pix_off + (long long)py * v.W + px;
  const long long p3 = 3 * v.pix_off + (long long)py * v.W + px;
  const float bg = b.p.bg;
  out.rgb[p3] = fmaf(T, bg, cr);
  out.rgb[p3 + HW] = fmaf(T, bg, cg);
  out.rgb[p3 + 2 * HW] = fmaf(T, bg, cb);
  out.normal[p3] = n0;
  out.normal[p3 + HW] = n1;
  out.normal[p3 + 2 * HW] = n2;
  // Eq. 7 with guards: |N . r| >= 1e-8 and accumulated weight >= 1e-6, else 0
  const float rx = fx_rel / v.fx, ry = fy_rel / v.fy;
  const float ndr = n0 * rx + n1 * ry + n2;
  const bool ok = fabsf(ndr) >= 1e-8f && (1.f - T) >= 1e-6f;
  out.depth[p] = ok ? D / ndr : 0.f;
  out.dist[p] = D;
  out.t_final[p] = T;
  out.last[p] = last;
  if (out.n_contrib) out.n_contrib[p] = ncontrib;
  if (out.n_eval) out.n_eval[p] = neval;
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

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) k_blend_bwd(const __grid_constant__ BatchDev b,
                                                       const float4* __restrict__ rec,
                                                       const uint32_t* __restrict__ pair_g,
                                                       const uint2* __restrict__ ranges, pgs_image_ptrs img,
                                                       pgs_image_grad_ptrs gi, float* __restrict__ grad) {
  constexpr int NT = TW * TH;
  __shared__ BlendSmem s;
  __shared__ float s_acc[NT][kGradFields];
  __shared__ uint32_t s_g[NT];
  __shared__ int s_max;
  const int tile = blockIdx.x;
  const uint2 rg = ranges[tile];
  if (rg.y <= rg.x) return;
  const int vi = view_of_tile(b, tile);
  const ViewDev& v = b.v[vi];
  const int lt = tile - v.tile_base;
  const int ty = lt / v.tiles_x, tx = lt - ty * v.tiles_x;
  const int px = tx * TW + (int)threadIdx.x % TW, py = ty * TH + (int)threadIdx.x / TW;
  const bool inside = px < v.W && py < v.H;
  const float fx_rel = (float)px + 0.5f - v.cx, fy_rel = (float)py + 0.5f - v.cy;
  const int lane = threadIdx.x & 31;
  const float a_min = b.p.alpha_min, a_max = b.p.alpha_max;

  uint32_t last = 0;
  float T = 1.f, gC0 = 0, gC1 = 0, gC2 = 0, gD = 0, gN0 = 0, gN1 = 0, gN2 = 0;
  float S0 = 0, S1 = 0, S2 = 0, SD = 0, SN0 = 0, SN1 = 0, SN2 = 0;
  if (inside) {
    const long long HW = (long long)v.W * v.H;
    const long long p = v.pix_off + (long long)py * v.W + px;
    const long long p3 = 3 * v.pix_off + (long long)py * v.W + px;
    last = img.last[p];
    T = img.t_final[p];
    gC0 = gi.rgb[p3]; gC1 = gi.rgb[p3 + HW]; gC2 = gi.rgb[p3 + 2 * HW];
    gN0 = gi.normal[p3]; gN1 = gi.normal[p3 + HW]; gN2 = gi.normal[p3 + 2 * HW];
    // chain through D_hat = D / (N . r)
    const float gDh = gi.depth[p];
    const float N0 = img.normal[p3], N1 = img.normal[p3 + HW], N2 = img.normal[p3 + 2 * HW];
    const float rx = fx_rel / v.fx, ry = fy_rel / v.fy;
    const float ndr = N0 * rx + N1 * ry + N2;
    const bool ok = fabsf(ndr) >= 1e-8f && (1.f - T) >= 1e-6f;
    if (ok) {
      const float D = img.dist[p];
      const float ind = 1.f / ndr;
      gD = gDh * ind;
      const float k = -gDh * D * ind * ind;
      gN0 += k * rx; gN1 += k * ry; gN2 += k;
    }
    const float bg = b.p.bg;
    S0 = S1 = S2 = T * bg;
  }
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  atomicMax(&s_max, (int)last);
  __syncthreads();
  const uint32_t end = (uint32_t)s_max;   // 1 + last contributor index over the tile
  for (uint32_t bend = end; bend > rg.x;) {
    const uint32_t bstart = bend > rg.x + NT ? bend - NT : rg.x;
    const int cnt = (int)(bend - bstart);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const uint32_t g = pair_g[bstart + threadIdx.x];
      s_g[threadIdx.x] = g;
      stage_record(s, threadIdx.x, rec, g);
#pragma unroll
      for (int f = 0; f < kGradFields; ++f) s_acc[threadIdx.x][f] = 0.f;
    }
    __syncthreads();
    // the warp walks from its highest live index down
    const int my_top = (int)min(last, bend) - 1 - (int)bstart;
    const int top = __reduce_max_sync(0xffffffffu, my_top);
    for (int k = top; k >= 0; --k) {
      const uint32_t j = bstart + k;
      bool contrib = false;
      float vals[16];
#pragma unroll
      for (int f = 0; f < 16; ++f) vals[f] = 0.f;
      if (j < last) {
        float dx, dy;
        const float4 q = s.q[k];
        const float power = eval_power(s.m[k], q, fx_rel, fy_rel, dx, dy);
        if (!(power > 0.f)) {
          const float a_raw = __fmul_rn(q.w, ex2_approx(power));
          if (!(a_raw < a_min)) {
            contrib = true;
            const float alpha = fminf(a_max, a_raw);
            const float om = __fsub_rn(1.f, alpha);
            const float iom = 1.f / om;
            T = T * iom;
            const float w = alpha * T;
            const float4 c = s.c[k], nn = s.n[k];
            const float dLda = gC0 * (c.x * T - S0 * iom) + gC1 * (c.y * T - S1 * iom) + gC2 * (c.z * T - S2 * iom) +
                               gD * (c.w * T - SD * iom) + gN0 * (nn.x * T - SN0 * iom) +
                               gN1 * (nn.y * T - SN1 * iom) + gN2 * (nn.z * T - SN2 * iom);
            S0 = fmaf(w, c.x, S0); S1 = fmaf(w, c.y, S1); S2 = fmaf(w, c.z, S2); SD = fmaf(w, c.w, SD);
            SN0 = fmaf(w, nn.x, SN0); SN1 = fmaf(w, nn.y, SN1); SN2 = fmaf(w, nn.z, SN2);
            vals[6] = w * gC0; vals[7] = w * gC1; vals[8] = w * gC2; vals[9] = w * gD;
            vals[10] = w * gN0; vals[11] = w * gN1; vals[12] = w * gN2;
            if (!(a_raw > a_max)) {
              // d alpha / d power_nat = a_raw ; natural conic = scaled / (-1/2 log2 e)
              const float G = dLda * a_raw;
              const float An = q.x * (1.f / kHalfLog2e), Bn = q.y * (1.f / kNegLog2e), Cn = q.z * (1.f / kHalfLog2e);
              vals[0] = G * (An * dx + Bn * dy);
              vals[1] = G * (Bn * dx + Cn * dy);
              vals[2] = -0.5f * G * dx * dx;
              vals[3] = -G * dx * dy;
              vals[4] = -0.5f * G * dy * dy;
              vals[5] = dLda * (a_raw / q.w);
            }
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        const float r = warp_transpose_reduce16(vals, lane);
        const int slot = (lane >> 1) & 15;
        if (!(lane & 1) && slot < kGradFields) atomicAdd(&s_acc[k][slot], r);
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const float* a = s_acc[threadIdx.x];
      float4* dst = reinterpret_cast<float4*>(grad + (size_t)s_g[threadIdx.x] * 16);
      const float4 v0 = make_float4(a[0], a[1], a[2], a[3]);
      const float4 v1 = make_float4(a[4], a[5], a[6], a[7]);
      const float4 v2 = make_float4(a[8], a[9], a[10], a[11]);
      if (v0.x != 0.f || v0.y != 0.f || v0.z != 0.f || v0.w != 0.f) atomicAdd(dst, v0);
      if (v1.x != 0.f || v1.y != 0.f || v1.z != 0.f || v1.w != 0.f) atomicAdd(dst + 1, v1);
      if (v2.x != 0.f || v2.y != 0.f || v2.z != 0.f || v2.w != 0.f) atomicAdd(dst + 2, v2);
      if (a[12] != 0.f) atomicAdd(reinterpret_cast<float*>(dst + 3), a[12]);
    }
    bend = bstart;
  }
}

template <int TW, int TH>
static void launch_fwd_t(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                         const pgs_image_ptrs& o, cudaStream_t st) {
  k_blend_fwd<TW, TH><<<b.total_tiles, TW * TH, 0, st>>>(b, rec, pg, rg, o);
}
template <int TW, int TH>
static void launch_bwd_t(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                         const pgs_image_ptrs& img, const pgs_image_grad_ptrs& gi, float* grad, cudaStream_t st) {
  k_blend_bwd<TW, TH><<<b.total_tiles, TW * TH, 0, st>>>(b, rec, pg, rg, img, gi, grad);
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
