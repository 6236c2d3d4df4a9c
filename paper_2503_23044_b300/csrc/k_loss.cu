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

// depth-derived normal at an interior pixel; false when not valid
__device__ __forceinline__ bool depth_normal(const BatchDev& b, const PixCtx& c, const float* __restrict__ depth,
                                             float nd[3]) {
  const ViewDev& v = b.v[c.v];
  if (c.px < 1 || c.py < 1 || c.px > v.W - 2 || c.py > v.H - 2) return false;
  const long long p = c.p;
  const float d0 = depth[p], dl = depth[p - 1], dr = depth[p + 1], du = depth[p - v.W], dd = depth[p + v.W];
  if (!(d0 > 0.f && dl > 0.f && dr > 0.f && du > 0.f && dd > 0.f)) return false;
  const float ifx = 1.f / v.fx, ify = 1.f / v.fy;
  const float u = (float)c.px + 0.5f - v.cx, w = (float)c.py + 0.5f - v.cy;
  // P = D_hat * ((u - cx)/fx, (v - cy)/fy, 1)
  const float ex0 = dr * (u + 1.f) * ifx - dl * (u - 1.f) * ifx, ex1 = (dr - dl) * w * ify, ex2 = dr - dl;
  const float ey0 = (dd - du) * u * ifx, ey1 = dd * (w + 1.f) * ify - du * (w - 1.f) * ify, ey2 = dd - du;
  float c0 = ex1 * ey2 - ex2 * ey1, c1 = ex2 * ey0 - ex0 * ey2, c2 = ex0 * ey1 - ex1 * ey0;
  const float nrm = sqrtf(c0 * c0 + c1 * c1 + c2 * c2);
  if (!(nrm > 1e-20f)) return false;
  const float in = 1.f / nrm;
  c0 *= in; c1 *= in; c2 *= in;
  const float face = c0 * d0 * u * ifx + c1 * d0 * w * ify + c2 * d0;
  if (face > 0.f) { c0 = -c0; c1 = -c1; c2 = -c2; }
  nd[0] = c0; nd[1] = c1; nd[2] = c2;
  return true;
}

__device__ __forceinline__ bool normal_valid(const BatchDev& b, const PixCtx& c, const pgs_image_ptrs& img, float nd[3],
                                             float N[3], float& nn) {
  if (!depth_normal(b, c, img.depth, nd)) return false;
  N[0] = img.normal[c.p3]; N[1] = img.normal[c.p3 + c.HW]; N[2] = img.normal[c.p3 + 2 * c.HW];
  nn = sqrtf(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  return nn > 1e-8f;
}

__device__ __forceinline__ void range_of_block(long long n, long long& s, long long& e) {
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  s = min(n, (long long)blockIdx.x * per);
  e = min(n, s + per);
}

__global__ void __launch_bounds__(256) k_loss_counts(const __grid_constant__ BatchDev b, pgs_image_ptrs img,
                                                     pgs_target_ptrs tgt, uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_cnt[kMaxViews][2];
  for (int i = threadIdx.x; i < kMaxViews * 2; i += blockDim.x) (&s_cnt[0][0])[i] = 0;
  __syncthreads();
  long long s, e;
  range_of_block(b.total_pixels, s, e);
  int vh = s < e ? view_of_pixel(b, s) : 0;
  for (long long p = s + threadIdx.x; p < e; p += blockDim.x) {
    const PixCtx c = pix_ctx(b, p, vh);
    float nd[3], N[3], nn;
    if (tgt.mask[p] > 0.f) atomicAdd(&s_cnt[c.v][0], 1u);
    if (normal_valid(b, c, img, nd, N, nn)) atomicAdd(&s_cnt[c.v][1], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kMaxViews * 2; i += blockDim.x)
    if ((&s_cnt[0][0])[i]) atomicAdd(counts + i, (&s_cnt[0][0])[i]);
}

__device__ __forceinline__ float sgnf(float x) { return (float)((x > 0.f) - (x < 0.f)); }

__global__ void __launch_bounds__(256) k_loss_grad(const __grid_constant__ BatchDev b, pgs_image_ptrs img,
                                                   pgs_target_ptrs tgt, pgs_loss_params lp,
                                                   const uint32_t* __restrict__ counts, pgs_image_grad_ptrs g,
                                                   float* __restrict__ partials, uint32_t* err) {
  __shared__ float s_red[3][256];
  long long s, e;
  range_of_block(b.total_pixels, s, e);
  const float invB = 1.f / (float)b.n_views;
  float l_rgb = 0.f, l_d = 0.f, l_n = 0.f;
  bool bad = false;
  int vh = s < e ? view_of_pixel(b, s) : 0;
  for (long long p = s + threadIdx.x; p < e; p += blockDim.x) {
    const PixCtx c = pix_ctx(b, p, vh);
    const float k_rgb = invB / (3.f * (float)c.HW);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const long long q = c.p3 + ch * c.HW;
      const float d = img.rgb[q] - tgt.rgb[q];
      l_rgb += fabsf(d) * k_rgb;
      g.rgb[q] = sgnf(d) * k_rgb;
    }
    const float mask = tgt.mask[p];
    float gd = 0.f;
    if (mask > 0.f) {
      const float kd = lp.lambda_depth * invB / fmaxf(1.f, (float)counts[2 * c.v]);
      const float d = img.depth[p] - tgt.prior[p];
      l_d += mask * fabsf(d) * kd;
      gd = mask * sgnf(d) * kd;
    }
    g.depth[p] = gd;
    float nd[3], N[3], nn, gn0 = 0.f, gn1 = 0.f, gn2 = 0.f;
    if (normal_valid(b, c, img, nd, N, nn)) {
      const float kn = lp.lambda_normal * invB / fmaxf(1.f, (float)counts[2 * c.v + 1]);
      const float inn = 1.f / nn;
      const float cosang = (nd[0] * N[0] + nd[1] * N[1] + nd[2] * N[2]) * inn;
      l_n += (1.f - cosang) * kn;
      // d/dN of -(N_d . N)/|N| = -(N_d/|N| - cos N/|N|^2)
      gn0 = -kn * (nd[0] * inn - cosang * N[0] * inn * inn);
      gn1 = -kn * (nd[1] * inn - cosang * N[1] * inn * inn);
      gn2 = -kn * (nd[2] * inn - cosang * N[2] * inn * inn);
    }
    g.normal[c.p3] = gn0;
    g.normal[c.p3 + c.HW] = gn1;
    g.normal[c.p3 + 2 * c.HW] = gn2;
    bad |= !isfinite(gd) || !isfinite(gn0) || !isfinite(gn1) || !isfinite(gn2);
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
  k_loss_counts<<<kLossBlocks, 256, 0, st>>>(b, img, tgt, counts);
  k_loss_grad<<<kLossBlocks, 256, 0, st>>>(b, img, tgt, lp, counts, g, partials, err);
  k_loss_final<<<1, 256, 0, st>>>(partials, kLossBlocks, loss, err);
}

}  // namespace pgs
