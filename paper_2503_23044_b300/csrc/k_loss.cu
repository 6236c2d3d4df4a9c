// Batch losses and their image gradients.
//   L = (1/B) sum_b [ mean|C_hat - I|                       (Eq. 8, mean over pixels and channels)
//                   + l_d * sum_mask |D_hat - D_prior| / |mask|       (Eq. 9)
//                   + l_n * mean_valid (1 - N_d . N_hat / |N_hat|) ]  (normal-depth consistency)
// N_d: normal of the surface implied by D_hat (cross product of the central
// differences of the back-projected neighbours, turned to face the camera),
// held constant (stop-gradient).  Valid pixels: interior, positive depth at
// the pixel and its four neighbours, |N_hat| > 1e-8.
// Sums are formed in a fixed order (per-thread ranges, per-block trees, one
// final block) so the loss value is reproducible run to run.
#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

struct PixCtx {
  int v, px, py;
  long long p, p3, HW;
};

// v is a running hint: threads walk increasing pixel indices, so the view only moves forward
__device__ __forceinline__ PixCtx pix_ctx(const BatchDev& b, long long p, int& v) {
  while (v + 1 < b.n_views && p >= b.v[v + 1].pix_off) ++v;
  PixCtx c;
  c.v = v;
  const ViewDev& vw = b.v[v];
  const unsigned l = (unsigned)(p - vw.pix_off);
  c.py = (int)(l / (unsigned)vw.W);
  c.px = (int)(l - (unsigned)c.py * (unsigned)vw.W);
  c.p = p;
  c.HW = (long long)vw.W * vw.H;
  c.p3 = 3 * vw.pix_off + l;
  return c;
}

// Inputs of one pixel, loaded before any arithmetic so that a thread keeps
// the loads of several pixels in flight (the loss is bound by HBM traffic).
struct PixIn {
  PixCtx c;
  bool inter;                 // interior pixel (the 5-point stencil exists)
  float d0, dl, dr, du, dd;   // D_hat at the pixel and its 4 neighbours
  float N[3];                 // N_hat
  float mask;
};

__device__ __forceinline__ void load_pix(const BatchDev& b, long long p, int& vh, const float* __restrict__ depth,
                                         const float* __restrict__ normal, const float* __restrict__ mask,
                                         PixIn& I) {
  I.c = pix_ctx(b, p, vh);
  const ViewDev& v = b.v[I.c.v];
  I.inter = I.c.px >= 1 && I.c.py >= 1 && I.c.px <= v.W - 2 && I.c.py <= v.H - 2;
  I.d0 = __ldg(depth + p);
  I.dl = I.dr = I.du = I.dd = 0.f;
  if (I.inter) {
    I.dl = __ldg(depth + p - 1); I.dr = __ldg(depth + p + 1);
    I.du = __ldg(depth + p - v.W); I.dd = __ldg(depth + p + v.W);
  }
  I.N[0] = __ldg(normal + I.c.p3); I.N[1] = __ldg(normal + I.c.p3 + I.c.HW); I.N[2] = __ldg(normal + I.c.p3 + 2 * I.c.HW);
  I.mask = __ldg(mask + p);
}

// depth-derived normal N_d (stop-gradient) and |N_hat|; false when the pixel is not valid
__device__ __forceinline__ bool normal_valid(const BatchDev& b, const PixIn& I, float nd[3], float& nn) {
  if (!I.inter) return false;
  if (!(I.d0 > 0.f && I.dl > 0.f && I.dr > 0.f && I.du > 0.f && I.dd > 0.f)) return false;
  const ViewDev& v = b.v[I.c.v];
  const float ifx = 1.f / v.fx, ify = 1.f / v.fy;
  const float u = (float)I.c.px + 0.5f - v.cx, w = (float)I.c.py + 0.5f - v.cy;
  // P = D_hat * ((u - cx)/fx, (v - cy)/fy, 1); N_d = normalised (dP/du x dP/dv), facing the camera
  const float dl = I.dl, dr = I.dr, du = I.du, dd = I.dd;
  const float ex0 = dr * (u + 1.f) * ifx - dl * (u - 1.f) * ifx, ex1 = (dr - dl) * w * ify, ex2 = dr - dl;
  const float ey0 = (dd - du) * u * ifx, ey1 = dd * (w + 1.f) * ify - du * (w - 1.f) * ify, ey2 = dd - du;
  float c0 = ex1 * ey2 - ex2 * ey1, c1 = ex2 * ey0 - ex0 * ey2, c2 = ex0 * ey1 - ex1 * ey0;
  const float nrm = sqrtf(c0 * c0 + c1 * c1 + c2 * c2);
  if (!(nrm > 1e-20f)) return false;
  const float in = 1.f / nrm;
  c0 *= in; c1 *= in; c2 *= in;
  const float face = c0 * I.d0 * u * ifx + c1 * I.d0 * w * ify + c2 * I.d0;
  if (face > 0.f) { c0 = -c0; c1 = -c1; c2 = -c2; }
  nd[0] = c0; nd[1] = c1; nd[2] = c2;
  nn = sqrtf(I.N[0] * I.N[0] + I.N[1] * I.N[1] + I.N[2] * I.N[2]);
  return nn > 1e-8f;
}

__device__ __forceinline__ void range_of_block(long long n, long long& s, long long& e) {
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  s = min(n, (long long)blockIdx.x * per);
  e = min(n, s + per);
}

constexpr int kCountUnroll = 4;  // pixels per thread per iteration, loads first
constexpr int kGradUnroll = 2;

// A thread's pixels run through the views in order, so it counts in registers for
// its current view and adds to the block's shared counters only when the view
// changes (integer sums: the result does not depend on the order).
struct ViewCounts {
  int v = -1;
  uint32_t c0 = 0, c1 = 0;
  __device__ __forceinline__ void flush(uint32_t (*s_cnt)[2]) {
    if (v >= 0) {
      if (c0) atomicAdd(&s_cnt[v][0], c0);
      if (c1) atomicAdd(&s_cnt[v][1], c1);
    }
    c0 = c1 = 0;
  }
  __device__ __forceinline__ void add(uint32_t (*s_cnt)[2], int pv, bool m, bool nv) {
    if (pv != v) {
      flush(s_cnt);
      v = pv;
    }
    c0 += m ? 1u : 0u;
    c1 += nv ? 1u : 0u;
  }
};

__global__ void __launch_bounds__(256) k_loss_counts(const __grid_constant__ BatchDev b, pgs_image_ptrs img,
                                                     pgs_target_ptrs tgt, uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_cnt[kMaxViews][2];
  for (int i = threadIdx.x; i < kMaxViews * 2; i += blockDim.x) (&s_cnt[0][0])[i] = 0;
  __syncthreads();
  const float* __restrict__ depth = img.depth;
  const float* __restrict__ normal = img.normal;
  const float* __restrict__ mask = tgt.mask;
  long long s, e;
  range_of_block(b.total_pixels, s, e);
  int vh = s < e ? view_of_pixel(b, s) : 0;
  ViewCounts vc;
  for (long long p0 = s + threadIdx.x; p0 < e; p0 += kCountUnroll * (long long)blockDim.x) {
    PixIn I[kCountUnroll];
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      const long long p = p0 + u * (long long)blockDim.x;
      if (p < e) load_pix(b, p, vh, depth, normal, mask, I[u]);
    }
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      const long long p = p0 + u * (long long)blockDim.x;
      if (p >= e) break;
      float nd[3], nn;
      vc.add(s_cnt, I[u].c.v, I[u].mask > 0.f, normal_valid(b, I[u], nd, nn));
    }
  }
  vc.flush(s_cnt);
  __syncthreads();
  for (int i = threadIdx.x; i < kMaxViews * 2; i += blockDim.x)
    if ((&s_cnt[0][0])[i]) atomicAdd(counts + i, (&s_cnt[0][0])[i]);
}

__device__ __forceinline__ float sgnf(float x) { return (float)((x > 0.f) - (x < 0.f)); }

__global__ void __launch_bounds__(256, 3) k_loss_grad(const __grid_constant__ BatchDev b, pgs_image_ptrs img,
                                                   pgs_target_ptrs tgt, pgs_loss_params lp,
                                                   const uint32_t* __restrict__ counts, pgs_image_grad_ptrs g,
                                                   float* __restrict__ partials, uint32_t* err) {
  __shared__ float s_red[3][256];
  const float* __restrict__ depth = img.depth;
  const float* __restrict__ normal = img.normal;
  const float* __restrict__ rgb = img.rgb;
  const float* __restrict__ trgb = tgt.rgb;
  const float* __restrict__ prior = tgt.prior;
  const float* __restrict__ mask = tgt.mask;
  float* __restrict__ g_rgb = g.rgb;
  float* __restrict__ g_depth = g.depth;
  float* __restrict__ g_normal = g.normal;
  long long s, e;
  range_of_block(b.total_pixels, s, e);
  const float invB = 1.f / (float)b.n_views;
  float l_rgb = 0.f, l_d = 0.f, l_n = 0.f;
  bool bad = false;
  int vh = s < e ? view_of_pixel(b, s) : 0;
  for (long long p0 = s + threadIdx.x; p0 < e; p0 += kGradUnroll * (long long)blockDim.x) {
    PixIn I[kGradUnroll];
    float c3[kGradUnroll][3], t3[kGradUnroll][3], pr[kGradUnroll];
#pragma unroll
    for (int u = 0; u < kGradUnroll; ++u) {
      const long long p = p0 + u * (long long)blockDim.x;
      if (p < e) {
        load_pix(b, p, vh, depth, normal, mask, I[u]);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          c3[u][ch] = __ldg(rgb + I[u].c.p3 + ch * I[u].c.HW);
          t3[u][ch] = __ldg(trgb + I[u].c.p3 + ch * I[u].c.HW);
        }
        pr[u] = __ldg(prior + p);
      }
    }
#pragma unroll
    for (int u = 0; u < kGradUnroll; ++u) {
      const long long p = p0 + u * (long long)blockDim.x;
      if (p >= e) break;
      const PixIn& P = I[u];
      const float k_rgb = invB / (3.f * (float)P.c.HW);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float d = c3[u][ch] - t3[u][ch];
        l_rgb += fabsf(d) * k_rgb;
        g_rgb[P.c.p3 + ch * P.c.HW] = sgnf(d) * k_rgb;
      }
      float gd = 0.f;
      if (P.mask > 0.f) {
        const float kd = lp.lambda_depth * invB / fmaxf(1.f, (float)counts[2 * P.c.v]);
        const float d = P.d0 - pr[u];
        l_d += P.mask * fabsf(d) * kd;
        gd = P.mask * sgnf(d) * kd;
      }
      g_depth[p] = gd;
      float nd[3], nn, gn0 = 0.f, gn1 = 0.f, gn2 = 0.f;
      if (normal_valid(b, P, nd, nn)) {
        const float kn = lp.lambda_normal * invB / fmaxf(1.f, (float)counts[2 * P.c.v + 1]);
        const float inn = 1.f / nn;
        const float cosang = (nd[0] * P.N[0] + nd[1] * P.N[1] + nd[2] * P.N[2]) * inn;
        l_n += (1.f - cosang) * kn;
        // d/dN of -(N_d . N)/|N| = -(N_d/|N| - cos N/|N|^2)
        gn0 = -kn * (nd[0] * inn - cosang * P.N[0] * inn * inn);
        gn1 = -kn * (nd[1] * inn - cosang * P.N[1] * inn * inn);
        gn2 = -kn * (nd[2] * inn - cosang * P.N[2] * inn * inn);
      }
      g_normal[P.c.p3] = gn0;
      g_normal[P.c.p3 + P.c.HW] = gn1;
      g_normal[P.c.p3 + 2 * P.c.HW] = gn2;
      bad |= !isfinite(gd) || !isfinite(gn0) || !isfinite(gn1) || !isfinite(gn2);
    }
  }
  if (bad) set_flag(err, kFlagNonfinite);
  s_red[0][threadIdx.x] = l_rgb;
  s_red[1][threadIdx.x] = l_d;
  s_red[2][threadIdx.x] = l_n;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int t = 0; t < 3; ++t) s_red[t][threadIdx.x] += s_red[t][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) partials[blockIdx.x * 3 + threadIdx.x] = s_red[threadIdx.x][0];
}

// ---------------------------------------------------------------- quad form
// When every view's width is a multiple of 4 and every map is 16-byte aligned,
// a thread takes 4 consecutive pixels of one row: each map is read and written
// with one 16-byte access per quad; the stencil's vertical neighbours come as
// two more 16-byte loads and the horizontal ones as two scalars.  The per-pixel
// arithmetic is the scalar form's (normal_valid and the loss terms below).
__device__ __forceinline__ float4 ld4(const float* __restrict__ p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float f4(const float4& v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w)); }
__device__ __forceinline__ void set4(float4& v, int i, float x) {
  if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
}

__device__ __forceinline__ void load_quad(const BatchDev& b, long long p, int& vh, const float* __restrict__ depth,
                                          const float* __restrict__ normal, const float* __restrict__ mask,
                                          PixIn (&I)[4]) {
  const PixCtx c = pix_ctx(b, p, vh);
  const ViewDev& v = b.v[c.v];
  const float4 d = ld4(depth + p);
  const bool rowin = c.py >= 1 && c.py <= v.H - 2;
  float4 up = make_float4(0.f, 0.f, 0.f, 0.f), dn = up;
  if (rowin) { up = ld4(depth + p - v.W); dn = ld4(depth + p + v.W); }
  const float left = c.px >= 1 ? __ldg(depth + p - 1) : 0.f;
  const float right = c.px + 4 <= v.W - 1 ? __ldg(depth + p + 4) : 0.f;
  const float4 n0 = ld4(normal + c.p3), n1 = ld4(normal + c.p3 + c.HW), n2 = ld4(normal + c.p3 + 2 * c.HW);
  const float4 m = ld4(mask + p);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    I[i].c = c;
    I[i].c.px = c.px + i;
    I[i].c.p = c.p + i;
    I[i].c.p3 = c.p3 + i;
    I[i].inter = rowin && c.px + i >= 1 && c.px + i <= v.W - 2;
    I[i].d0 = f4(d, i);
    I[i].dl = i == 0 ? left : f4(d, i - 1);
    I[i].dr = i == 3 ? right : f4(d, i + 1);
    I[i].du = f4(up, i);
    I[i].dd = f4(dn, i);
    I[i].N[0] = f4(n0, i); I[i].N[1] = f4(n1, i); I[i].N[2] = f4(n2, i);
    I[i].mask = f4(m, i);
  }
}

__global__ void __launch_bounds__(256) k_loss_counts4(const __grid_constant__ BatchDev b, pgs_image_ptrs img,
                                                      pgs_target_ptrs tgt, uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_cnt[kMaxViews][2];
  for (int i = threadIdx.x; i < kMaxViews * 2; i += blockDim.x) (&s_cnt[0][0])[i] = 0;
  __syncthreads();
  long long s, e;
  range_of_block(b.total_pixels / 4, s, e);
  int vh = s < e ? view_of_pixel(b, 4 * s) : 0;
  ViewCounts vc;
  for (long long q0 = s + threadIdx.x; q0 < e; q0 += 2 * (long long)blockDim.x) {
    PixIn I[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const long long q = q0 + u * (long long)blockDim.x;
      if (q < e) load_quad(b, 4 * q, vh, img.depth, img.normal, tgt.mask, I[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (q0 + u * (long long)blockDim.x >= e) break;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float nd[3], nn;
        vc.add(s_cnt, I[u][i].c.v, I[u][i].mask > 0.f, normal_valid(b, I[u][i], nd, nn));
      }
    }
  }
  vc.flush(s_cnt);
  __syncthreads();
  for (int i = threadIdx.x; i < kMaxViews * 2; i += blockDim.x)
    if ((&s_cnt[0][0])[i]) atomicAdd(counts + i, (&s_cnt[0][0])[i]);
}

__global__ void __launch_bounds__(256) k_loss_grad4(const __grid_constant__ BatchDev b, pgs_image_ptrs img,
                                                    pgs_target_ptrs tgt, pgs_loss_params lp,
                                                    const uint32_t* __restrict__ counts, pgs_image_grad_ptrs g,
                                                    float* __restrict__ partials, uint32_t* err) {
  __shared__ float s_red[3][256];
  long long s, e;
  range_of_block(b.total_pixels / 4, s, e);
  const float invB = 1.f / (float)b.n_views;
  float l_rgb = 0.f, l_d = 0.f, l_n = 0.f;
  bool bad = false;
  int vh = s < e ? view_of_pixel(b, 4 * s) : 0;
  for (long long q = s + threadIdx.x; q < e; q += blockDim.x) {
    const long long p = 4 * q;
    PixIn I[4];
    load_quad(b, p, vh, img.depth, img.normal, tgt.mask, I);
    const PixCtx& c = I[0].c;
    float4 c3[3], t3[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      c3[ch] = ld4(img.rgb + c.p3 + ch * c.HW);
      t3[ch] = ld4(tgt.rgb + c.p3 + ch * c.HW);
    }
    const float4 pr = ld4(tgt.prior + p);
    const float k_rgb = invB / (3.f * (float)c.HW);
    const float kd = lp.lambda_depth * invB / fmaxf(1.f, (float)counts[2 * c.v]);
    const float kn = lp.lambda_normal * invB / fmaxf(1.f, (float)counts[2 * c.v + 1]);
    float4 grgb[3], gdep, gnor[3];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float d = f4(c3[ch], i) - f4(t3[ch], i);
        l_rgb += fabsf(d) * k_rgb;
        set4(grgb[ch], i, sgnf(d) * k_rgb);
      }
      const PixIn& P = I[i];
      float gd = 0.f;
      if (P.mask > 0.f) {
        const float d = P.d0 - f4(pr, i);
        l_d += P.mask * fabsf(d) * kd;
        gd = P.mask * sgnf(d) * kd;
      }
      set4(gdep, i, gd);
      float nd[3], nn, gn0 = 0.f, gn1 = 0.f, gn2 = 0.f;
      if (normal_valid(b, P, nd, nn)) {
        const float inn = 1.f / nn;
        const float cosang = (nd[0] * P.N[0] + nd[1] * P.N[1] + nd[2] * P.N[2]) * inn;
        l_n += (1.f - cosang) * kn;
        gn0 = -kn * (nd[0] * inn - cosang * P.N[0] * inn * inn);
        gn1 = -kn * (nd[1] * inn - cosang * P.N[1] * inn * inn);
        gn2 = -kn * (nd[2] * inn - cosang * P.N[2] * inn * inn);
      }
      set4(gnor[0], i, gn0); set4(gnor[1], i, gn1); set4(gnor[2], i, gn2);
      bad |= !isfinite(gd) || !isfinite(gn0) || !isfinite(gn1) || !isfinite(gn2);
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      *reinterpret_cast<float4*>(g.rgb + c.p3 + ch * c.HW) = grgb[ch];
      *reinterpret_cast<float4*>(g.normal + c.p3 + ch * c.HW) = gnor[ch];
    }
    *reinterpret_cast<float4*>(g.depth + p) = gdep;
  }
  if (bad) set_flag(err, kFlagNonfinite);
  s_red[0][threadIdx.x] = l_rgb;
  s_red[1][threadIdx.x] = l_d;
  s_red[2][threadIdx.x] = l_n;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int t = 0; t < 3; ++t) s_red[t][threadIdx.x] += s_red[t][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) partials[blockIdx.x * 3 + threadIdx.x] = s_red[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) k_loss_final(const float* __restrict__ partials, int nb, float* __restrict__ loss,
                                                    uint32_t* err) {
  __shared__ float s_red[3][256];
  float a[3] = {0.f, 0.f, 0.f};
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    for (int t = 0; t < 3; ++t) a[t] += partials[i * 3 + t];
  for (int t = 0; t < 3; ++t) s_red[t][threadIdx.x] = a[t];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int t = 0; t < 3; ++t) s_red[t][threadIdx.x] += s_red[t][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float tot = s_red[0][0] + s_red[1][0] + s_red[2][0];
    loss[0] = tot;
    loss[1] = s_red[0][0];
    loss[2] = s_red[1][0];
    loss[3] = s_red[2][0];
    if (!isfinite(tot)) set_flag(err, kFlagNonfinite);
  }
}

void launch_loss(const BatchDev& b, const pgs_image_ptrs& img, const pgs_target_ptrs& tgt, const pgs_loss_params& lp,
                 float* loss, const pgs_image_grad_ptrs& g, uint32_t* counts, float* partials, uint32_t* err,
                 cudaStream_t st) {
  cudaMemsetAsync(counts, 0, kMaxViews * 2 * sizeof(uint32_t), st);
  bool quad = true;
  for (int v = 0; v < b.n_views; ++v) quad = quad && b.v[v].W % 4 == 0;
  for (const void* ptr : {(const void*)img.rgb, (const void*)img.depth, (const void*)img.normal, (const void*)tgt.rgb,
                          (const void*)tgt.prior, (const void*)tgt.mask, (const void*)g.rgb, (const void*)g.depth,
                          (const void*)g.normal})
    quad = quad && (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0;
  if (quad) {
    k_loss_counts4<<<kLossBlocks, 256, 0, st>>>(b, img, tgt, counts);
    k_loss_grad4<<<kLossBlocks, 256, 0, st>>>(b, img, tgt, lp, counts, g, partials, err);
  } else {
    k_loss_counts<<<kLossBlocks, 256, 0, st>>>(b, img, tgt, counts);
    k_loss_grad<<<kLossBlocks, 256, 0, st>>>(b, img, tgt, lp, counts, g, partials, err);
  }
  k_loss_final<<<1, 256, 0, st>>>(partials, kLossBlocks, loss, err);
}

}  // namespace pgs
