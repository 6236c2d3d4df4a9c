// Enhanced depth prior (Step 2 of the batch-level progressive training, Sec. 3.4;
// tau_d = 1 in the supplementary implementation details).
//
// 1. Scale and shift: per view v, least squares of the sparse points' view
//    depths z_k against the pseudo depth D_p sampled (bilinear) where they
//    project: (s_v, t_v) = argmin sum_k (s D_p(u_k) + t - z_k)^2, so
//    D~_p = s_v D_p + t_v has the points' scale.  Two passes (means, then
//    centred sums) keep the FP32 normal equations well conditioned; every sum is
//    formed in a fixed order.
// 2. Re-projection error: pixel p of view a, at depth D~_p,a(p), is lifted to 3D,
//    projected into each of its k nearest batch views b (by camera centre), where
//    D~_p,b is read (bilinear) and lifted again; that point is projected back
//    into a, and e_b = |p' - p| in pixels.  E(p) = min over the neighbours whose
//    round trip is defined (in front of both cameras, inside b's frame, a prior
//    at all four samples).
// 3. Filter: D~_f(p) = D~_p(p) where E(p) <= tau_d, or where no neighbour could
//    check p; 0 where E(p) > tau_d or the prior is missing.  The mask is the
//    depth L1 mask of the loss.
#include <algorithm>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

// pseudo depth at continuous pixel coordinates (pixel centres at +0.5); false
// outside the frame or when one of the four samples has no prior (<= 0)
__device__ __forceinline__ bool prior_bilinear(const float* __restrict__ dp, const ViewDev& v, float x, float y,
                                               float& out) {
  const float u = x - 0.5f, w = y - 0.5f;
  const float fu = floorf(u), fw = floorf(w);
  if (!(fu >= 0.f && fw >= 0.f && fu + 1.f <= (float)(v.W - 1) && fw + 1.f <= (float)(v.H - 1))) return false;
  const int i0 = (int)fu, j0 = (int)fw;
  const float au = u - fu, aw = w - fw;
  const float* r0 = dp + v.pix_off + (long long)j0 * v.W + i0;
  const float* r1 = r0 + v.W;
  const float a = __ldg(r0), b = __ldg(r0 + 1), c = __ldg(r1), d = __ldg(r1 + 1);
  if (!(a > 0.f && b > 0.f && c > 0.f && d > 0.f)) return false;
  const float top = fmaf(au, b - a, a), bot = fmaf(au, d - c, c);
  out = fmaf(aw, bot - top, top);
  return true;
}

__device__ __forceinline__ void to_cam(const ViewDev& v, const float x[3], float c[3]) {
  c[0] = v.R[0] * x[0] + v.R[1] * x[1] + v.R[2] * x[2] + v.t[0];
  c[1] = v.R[3] * x[0] + v.R[4] * x[1] + v.R[5] * x[2] + v.t[1];
  c[2] = v.R[6] * x[0] + v.R[7] * x[1] + v.R[8] * x[2] + v.t[2];
}
// world point of camera-frame point c: R^T (c - t)
__device__ __forceinline__ void to_world(const ViewDev& v, const float c[3], float x[3]) {
  const float a = c[0] - v.t[0], b = c[1] - v.t[1], d = c[2] - v.t[2];
  x[0] = v.R[0] * a + v.R[3] * b + v.R[6] * d;
  x[1] = v.R[1] * a + v.R[4] * b + v.R[7] * d;
  x[2] = v.R[2] * a + v.R[5] * b + v.R[8] * d;
}

// pass 0: (n, sum d, sum z); pass 1: (sum (d - dm)^2, sum (d - dm)(z - zm), 0) per (view, block)
__global__ void __launch_bounds__(256) k_prior_fit_partial(const __grid_constant__ BatchDev b,
                                                           const float* __restrict__ dp,
                                                           const float* __restrict__ pts, long long n_pts, int pass,
                                                           const float* __restrict__ means,
                                                           float* __restrict__ partials) {
  __shared__ float s_red[3][256];
  const int vi = blockIdx.y;
  const ViewDev& v = b.v[vi];
  const float dm = pass ? means[vi * 4 + 1] : 0.f, zm = pass ? means[vi * 4 + 2] : 0.f;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_pts;
       k += (long long)gridDim.x * blockDim.x) {
    const float x[3] = {pts[3 * k], pts[3 * k + 1], pts[3 * k + 2]};
    float c[3];
    to_cam(v, x, c);
    if (!(c[2] > b.p.near_plane)) continue;
    const float px = v.fx * c[0] / c[2] + v.cx, py = v.fy * c[1] / c[2] + v.cy;
    float d;
    if (!prior_bilinear(dp, v, px, py, d)) continue;
    if (pass == 0) { a0 += 1.f; a1 += d; a2 += c[2]; }
    else { const float dd = d - dm; a0 = fmaf(dd, dd, a0); a1 = fmaf(dd, c[2] - zm, a1); }
  }
  s_red[0][threadIdx.x] = a0;
  s_red[1][threadIdx.x] = a1;
  s_red[2][threadIdx.x] = a2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int t = 0; t < 3; ++t) s_red[t][threadIdx.x] += s_red[t][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) partials[((long long)vi * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = s_red[threadIdx.x][0];
}

// one thread per view, partials added in block order.  pass 0 -> means[v] = (n, dm, zm, -);
// pass 1 -> scale_shift[v] = (s, t); with fewer than 2 points or no spread: (1, 0) and n stored as 0
__global__ void k_prior_fit_final(const float* __restrict__ partials, int nb, int n_views, int pass,
                                  float* __restrict__ means, float* __restrict__ scale_shift) {
  const int vi = threadIdx.x;
  if (vi >= n_views) return;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (int k = 0; k < nb; ++k) {
    const float* q = partials + ((long long)vi * nb + k) * 3;
    a0 += q[0]; a1 += q[1]; a2 += q[2];
  }
  if (pass == 0) {
    means[vi * 4 + 0] = a0;
    means[vi * 4 + 1] = a0 > 0.f ? a1 / a0 : 0.f;
    means[vi * 4 + 2] = a0 > 0.f ? a2 / a0 : 0.f;
    means[vi * 4 + 3] = 0.f;
  } else {
    const float n = means[vi * 4 + 0];
    const bool ok = n >= 2.f && a0 > 1e-12f * n;
    const float s = ok ? a1 / a0 : 1.f;
    scale_shift[2 * vi] = s;
    scale_shift[2 * vi + 1] = ok ? means[vi * 4 + 2] - s * means[vi * 4 + 1] : 0.f;
  }
}

// Bilinear footprint of continuous pixel coordinates (x, y) in view v: the
// address of the top-left sample and the weights; false outside the frame.
// prior_bilinear split in two so that a thread can issue the loads of every
// neighbour view before it uses any of them.
__device__ __forceinline__ bool prior_footprint(const ViewDev& v, float x, float y, long long& at, float& au,
                                                float& aw) {
  const float u = x - 0.5f, w = y - 0.5f;
  const float fu = floorf(u), fw = floorf(w);
  if (!(fu >= 0.f && fw >= 0.f && fu + 1.f <= (float)(v.W - 1) && fw + 1.f <= (float)(v.H - 1))) return false;
  at = v.pix_off + (long long)(int)fw * v.W + (int)fu;
  au = u - fu;
  aw = w - fw;
  return true;
}

// One thread per pixel at a time (grid-stride).  The pixel's own pseudo depth is
// loaded one iteration ahead, and the k neighbour views are taken in two phases
// (project and issue the four loads of every neighbour, then finish the round
// trips), so the gathers of a pixel are in flight together; the arithmetic of
// each neighbour and the order of the minimum are those of the definition above.
// K = pa.k, the number of neighbour views (0..kPriorMaxK), fixed per launch.
template <int K>
__global__ void __launch_bounds__(256) k_prior_filter(const __grid_constant__ BatchDev b, PriorArgs pa,
                                                      const float* __restrict__ dp,
                                                      const float* __restrict__ scale_shift,
                                                      float* __restrict__ prior_out, float* __restrict__ mask_out,
                                                      float* __restrict__ err_out) {
  // the batch's view parameters, scale/shift pairs and neighbour lists, read at data-dependent
  // indices for every pixel, are copied once per CTA into shared memory
  __shared__ ViewDev s_v[kMaxViews];
  __shared__ float s_ss[2 * kMaxViews];
  __shared__ int s_nbr[kMaxViews][K + 1];
  {
    const int nw = b.n_views * (int)(sizeof(ViewDev) / sizeof(uint32_t));
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&b.v[0]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s_v[0]);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < 2 * b.n_views; i += blockDim.x) s_ss[i] = scale_shift[i];
    if constexpr (K > 0)
      for (int i = threadIdx.x; i < b.n_views * K; i += blockDim.x) s_nbr[i / K][i % K] = pa.nbr[i / K][i % K];
  }
  __syncthreads();
  int vi = 0;   // threads walk increasing pixel indices, so the view only moves forward
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float raw_next = p < b.total_pixels ? __ldg(dp + p) : 0.f;
  for (; p < b.total_pixels; p += stride) {
    const float raw = raw_next;
    raw_next = p + stride < b.total_pixels ? __ldg(dp + p + stride) : 0.f;
    while (vi + 1 < b.n_views && p >= s_v[vi + 1].pix_off) ++vi;
    const ViewDev& va = s_v[vi];
    const unsigned l = (unsigned)(p - va.pix_off);
    const int py = (int)(l / (unsigned)va.W), px = (int)(l - (unsigned)py * (unsigned)va.W);
    const float d = fmaf(s_ss[2 * vi], raw, s_ss[2 * vi + 1]);
    float keep_d = 0.f, keep = 0.f, E = -1.f;
    if (raw > 0.f && d > 0.f) {
      const float ux = (float)px + 0.5f, uy = (float)py + 0.5f;
      const float ca[3] = {d * (ux - va.cx) * rcp_approx(va.fx), d * (uy - va.cy) * rcp_approx(va.fy), d};
      float xw[3];
      to_world(va, ca, xw);
      // phase 1: every neighbour's projection and its four samples
      float qx[K + 1], qy[K + 1], au[K + 1], aw[K + 1], sm[K + 1][4];
      bool ok[K + 1];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        ok[i] = false;
        qx[i] = qy[i] = au[i] = aw[i] = 0.f;
        sm[i][0] = sm[i][1] = sm[i][2] = sm[i][3] = 0.f;
        const int nb = s_nbr[vi][i];
        if (nb < 0) continue;
        const ViewDev& vb = s_v[nb];
        float cb[3];
        to_cam(vb, xw, cb);
        if (!(cb[2] > b.p.near_plane)) continue;
        const float izb = rcp_approx(cb[2]);
        qx[i] = fmaf(vb.fx * cb[0], izb, vb.cx);
        qy[i] = fmaf(vb.fy * cb[1], izb, vb.cy);
        long long at;
        if (!prior_footprint(vb, qx[i], qy[i], at, au[i], aw[i])) continue;
        const float* r0 = dp + at;
        sm[i][0] = __ldg(r0); sm[i][1] = __ldg(r0 + 1); sm[i][2] = __ldg(r0 + vb.W); sm[i][3] = __ldg(r0 + vb.W + 1);
        ok[i] = true;
      }
      // phase 2: the round trips back into view a, in neighbour order
      float best = 3.4e38f;
      bool checked = false;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        if (!ok[i]) continue;
        const float a = sm[i][0], bb = sm[i][1], c = sm[i][2], dd = sm[i][3];
        if (!(a > 0.f && bb > 0.f && c > 0.f && dd > 0.f)) continue;
        const float top = fmaf(au[i], bb - a, a), bot = fmaf(au[i], dd - c, c);
        const float rb = fmaf(aw[i], bot - top, top);
        const int nb = s_nbr[vi][i];
        const ViewDev& vb = s_v[nb];
        const float db = fmaf(s_ss[2 * nb], rb, s_ss[2 * nb + 1]);
        if (!(db > 0.f)) continue;
        const float cb2[3] = {db * (qx[i] - vb.cx) * rcp_approx(vb.fx), db * (qy[i] - vb.cy) * rcp_approx(vb.fy), db};
        float xw2[3], ca2[3];
        to_world(vb, cb2, xw2);
        to_cam(va, xw2, ca2);
        if (!(ca2[2] > b.p.near_plane)) continue;
        const float iza = rcp_approx(ca2[2]);
        const float rx = fmaf(va.fx * ca2[0], iza, va.cx) - ux, ry = fmaf(va.fy * ca2[1], iza, va.cy) - uy;
        best = fminf(best, sqrtf(rx * rx + ry * ry));
        checked = true;
      }
      if (checked) E = best;
      if (!checked || best <= pa.tau_d) { keep_d = d; keep = 1.f; }
    }
    prior_out[p] = keep_d;
    mask_out[p] = keep;
    if (err_out) err_out[p] = E;
  }
}

void launch_prior_filter(const BatchDev& b, const PriorArgs& pa, const float* dp, const float* pts, long long n_pts,
                         float* partials, float* means, float* scale_shift, float* prior_out, float* mask_out,
                         float* err_out, int num_sms, cudaStream_t st) {
  const dim3 g(kPriorBlocks, b.n_views);
  for (int pass = 0; pass < 2; ++pass) {
    k_prior_fit_partial<<<g, 256, 0, st>>>(b, dp, pts, n_pts, pass, means, partials);
    k_prior_fit_final<<<1, kMaxViews, 0, st>>>(partials, kPriorBlocks, b.n_views, pass, means, scale_shift);
  }
  // one resident wave of the variant for this neighbour count
  auto filter = [&](auto kernel) {
    const int fg = std::max(1, resident_ctas_per_sm(reinterpret_cast<const void*>(kernel), 256)) * num_sms;
    kernel<<<fg, 256, 0, st>>>(b, pa, dp, scale_shift, prior_out, mask_out, err_out);
  };
  switch (pa.k) {
    case 0: filter(k_prior_filter<0>); break;
    case 1: filter(k_prior_filter<1>); break;
    case 2: filter(k_prior_filter<2>); break;
    case 3: filter(k_prior_filter<3>); break;
    default: filter(k_prior_filter<kPriorMaxK>);
  }
}

}  // namespace pgs
