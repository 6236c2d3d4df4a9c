// Batch geometric NCC loss (Step 3 of the batch-level progressive training,
// Sec. 3.4, Eq. 10).
//
// The batch is split into pairs; pair i has the reference view r = 2i+1 and the
// partner s = 2i (0-based).  For each drawn centre p of r, the 7 x 7 patch of
// reference pixels is mapped into s by the homography of the plane through the
// back-projected centre: m . X = 1 with m = N_hat(p) / (D_hat(p) (N_hat(p) . r_p)),
// r_p = K_r^-1 p~, so reference pixel q lands where R_sr r_q + t_sr (m . r_q)
// projects in s (X_s = R_sr X_r + t_sr; this is K_s (R_sr + t_sr m^T) K_r^-1 q~
// without forming the 3 x 3 product).  NCC compares the BT.601 luma of the
// reference pixels with the partner's luma read bilinearly at the warped
// positions: NCC = S_ab / sqrt((S_aa + eps)(S_bb + eps)) over centred sums.
// L_ncc = (1 / (B/2)) sum_i mean over pair i's valid patches of (1 - NCC).
//
// Stop-gradient (sg[.] of Eq. 10): the partner's colours are constants.  In the
// geometric form the warped positions keep their dependence on D_hat(p) and
// N_hat(p), so dL/dD_hat and dL/dN_hat at each centre come through the bilinear
// slope of the partner's luma; in the literal form only the reference colours
// receive gradients.
//
// Four kernels: the luma of every paired view and the pairs' relative poses
// (one pass over the pixels); validity and per-pair counts (one thread per
// patch, integer atomics so the counts are exact); the patch pass (one warp per
// used patch: NCC, gradients scaled by the now known 1 / count, float atomics
// into the image gradients); and a fixed-order reduction of the loss (one block
// per pair, the last block to finish adds the pairs in order).
//
// Validity is tested on the four corner samples of a patch: the plane factor
// m . r_q and the partner depth are affine in the pixel coordinate, so they are
// positive on the whole patch iff they are at its corners, and the warp is then
// a projective map that takes the square to a convex quadrilateral, which lies
// in the (convex) bilinear footprint area iff its corners do.
#include <algorithm>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

namespace {

constexpr int kHalf = 3, kSide = 7, kTaps = kSide * kSide;
constexpr float kLumaR = 0.299f, kLumaG = 0.587f, kLumaB = 0.114f;

// relative pose of a pair, X_s = R X_r + t, written once per call by k_ncc_luma
struct PairGeo {
  float R[9], t[3];
};

__device__ __forceinline__ void pair_geo(const ViewDev& vr, const ViewDev& vs, PairGeo& g) {
  // R = R_s R_r^T, t = t_s - R t_r
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      g.R[3 * i + j] = fmaf(vs.R[3 * i + 0], vr.R[3 * j + 0],
                            fmaf(vs.R[3 * i + 1], vr.R[3 * j + 1], vs.R[3 * i + 2] * vr.R[3 * j + 2]));
#pragma unroll
  for (int i = 0; i < 3; ++i)
    g.t[i] = vs.t[i] - fmaf(g.R[3 * i + 0], vr.t[0], fmaf(g.R[3 * i + 1], vr.t[1], g.R[3 * i + 2] * vr.t[2]));
}

// the patch centre: plane vector m, the centre ray r_p and the inputs the
// gradient needs; false when the patch is not usable
struct Centre {
  int x, y;
  long long p;           // arena index of the centre pixel
  float d, n[3], rp[3], c, m[3], ifx, ify;
};

// the centre's position; false when its patch leaves the reference frame
__device__ __forceinline__ bool centre_pos(const ViewDev& vr, unsigned cidx, Centre& C) {
  if ((long long)cidx >= (long long)vr.W * vr.H) return false;
  C.y = (int)(cidx / (unsigned)vr.W);
  C.x = (int)(cidx - (unsigned)C.y * (unsigned)vr.W);
  if (C.x < kHalf || C.y < kHalf || C.x > vr.W - 1 - kHalf || C.y > vr.H - 1 - kHalf) return false;
  C.p = vr.pix_off + cidx;
  return true;
}

// D_hat and N_hat at the centre
__device__ __forceinline__ void centre_fetch(const ViewDev& vr, const Centre& C, const float* __restrict__ depth,
                                             const float* __restrict__ normal, float& d, float n[3]) {
  const long long HW = (long long)vr.W * vr.H;
  const long long p3 = 2 * vr.pix_off + C.p;
  d = __ldg(depth + C.p);
  n[0] = __ldg(normal + p3);
  n[1] = __ldg(normal + p3 + HW);
  n[2] = __ldg(normal + p3 + 2 * HW);
}

// the plane of the centre; false when it is not defined
__device__ __forceinline__ bool centre_plane(const ViewDev& vr, float d, const float n[3], Centre& C) {
  C.d = d;
  C.n[0] = n[0];
  C.n[1] = n[1];
  C.n[2] = n[2];
  C.ifx = rcp_approx(vr.fx);
  C.ify = rcp_approx(vr.fy);
  C.rp[0] = ((float)C.x + 0.5f - vr.cx) * C.ifx;
  C.rp[1] = ((float)C.y + 0.5f - vr.cy) * C.ify;
  C.rp[2] = 1.f;
  C.c = fmaf(C.n[0], C.rp[0], fmaf(C.n[1], C.rp[1], C.n[2]));
  if (!(C.d > 0.f) || !(fabsf(C.c) >= 1e-8f)) return false;
  const float iden = rcp_approx(C.d * C.c);
  C.m[0] = C.n[0] * iden;
  C.m[1] = C.n[1] * iden;
  C.m[2] = C.n[2] * iden;
  return true;
}

// warped position of the sample at offset (dx, dy) from the centre; rq: its
// reference ray, P: partner camera coordinates up to the positive factor m . r_q
struct Warp {
  float rq[2], mr, P[3], iz, u, v;
};

__device__ __forceinline__ void warp_sample(const ViewDev& vs, const PairGeo& g, const Centre& C, int dx, int dy,
                                            Warp& w) {
  w.rq[0] = fmaf((float)dx, C.ifx, C.rp[0]);
  w.rq[1] = fmaf((float)dy, C.ify, C.rp[1]);
  w.mr = fmaf(C.m[0], w.rq[0], fmaf(C.m[1], w.rq[1], C.m[2]));
#pragma unroll
  for (int i = 0; i < 3; ++i)
    w.P[i] = fmaf(g.t[i], w.mr, fmaf(g.R[3 * i + 0], w.rq[0], fmaf(g.R[3 * i + 1], w.rq[1], g.R[3 * i + 2])));
  w.iz = rcp_approx(w.P[2]);
  w.u = fmaf(vs.fx * w.P[0], w.iz, vs.cx);
  w.v = fmaf(vs.fy * w.P[1], w.iz, vs.cy);
}

// the sample has the plane in front of both cameras and its bilinear footprint
// (pixel centres at +1/2) inside the partner frame
__device__ __forceinline__ bool sample_ok(const ViewDev& vs, const Warp& w) {
  if (!(w.mr > 0.f && w.P[2] > 0.f)) return false;
  const float fu = floorf(w.u - 0.5f), fv = floorf(w.v - 0.5f);
  return fu >= 0.f && fv >= 0.f && fu + 1.f <= (float)(vs.W - 1) && fv + 1.f <= (float)(vs.H - 1);
}

// partner luma, bilinear at (u, v), and its slope (du, dv); indices clamped so
// that the reads stay inside the view whatever the rounding of the position
__device__ __forceinline__ float luma_bilinear(const ViewDev& vs, const float* __restrict__ luma, float u, float v,
                                               float& gu, float& gv) {
  const float x = u - 0.5f, y = v - 0.5f;
  const float fx = floorf(x), fy = floorf(y);
  const int i0 = min(max((int)fx, 0), vs.W - 2), j0 = min(max((int)fy, 0), vs.H - 2);
  const float ax = x - fx, ay = y - fy;
  const float* q = luma + vs.pix_off + (j0 * vs.W + i0);
  const float g00 = __ldg(q), g10 = __ldg(q + 1), g01 = __ldg(q + vs.W), g11 = __ldg(q + vs.W + 1);
  const float top = fmaf(ax, g10 - g00, g00), bot = fmaf(ax, g11 - g01, g01);
  gu = fmaf(ay, (g11 - g01) - (g10 - g00), g10 - g00);
  gv = bot - top;
  return fmaf(ay, bot - top, top);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

}  // namespace

// pass 0: BT.601 luma of the paired views' colour (the first n_pix pixels of the
// arena) and the pairs' relative poses
__global__ void __launch_bounds__(256) k_ncc_luma(const __grid_constant__ BatchDev b, int n_pairs,
                                                  const float* __restrict__ rgb, long long n_pix, bool quad,
                                                  float* __restrict__ luma, PairGeo* __restrict__ geo) {
  if (blockIdx.x == 0 && (int)threadIdx.x < n_pairs) {
    PairGeo g;
    pair_geo(b.v[2 * threadIdx.x + 1], b.v[2 * threadIdx.x], g);
    geo[threadIdx.x] = g;
  }
  int v = 0;
  if (quad) {   // every view's pixel count and offset a multiple of 4, 16-byte aligned maps
    for (long long p = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x); p < n_pix;
         p += 4 * (long long)gridDim.x * blockDim.x) {
      while (v + 1 < b.n_views && p >= b.v[v + 1].pix_off) ++v;
      const ViewDev& w = b.v[v];
      const long long HW = (long long)w.W * w.H;
      const long long p3 = 3 * w.pix_off + (p - w.pix_off);
      const float4 r = __ldg(reinterpret_cast<const float4*>(rgb + p3));
      const float4 g = __ldg(reinterpret_cast<const float4*>(rgb + p3 + HW));
      const float4 c = __ldg(reinterpret_cast<const float4*>(rgb + p3 + 2 * HW));
      float4 y;
      y.x = fmaf(kLumaR, r.x, fmaf(kLumaG, g.x, kLumaB * c.x));
      y.y = fmaf(kLumaR, r.y, fmaf(kLumaG, g.y, kLumaB * c.y));
      y.z = fmaf(kLumaR, r.z, fmaf(kLumaG, g.z, kLumaB * c.z));
      y.w = fmaf(kLumaR, r.w, fmaf(kLumaG, g.w, kLumaB * c.w));
      *reinterpret_cast<float4*>(luma + p) = y;
    }
    return;
  }
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n_pix;
       p += (long long)gridDim.x * blockDim.x) {
    while (v + 1 < b.n_views && p >= b.v[v + 1].pix_off) ++v;
    const ViewDev& w = b.v[v];
    const long long HW = (long long)w.W * w.H;
    const long long p3 = 3 * w.pix_off + (p - w.pix_off);
    luma[p] = fmaf(kLumaR, __ldg(rgb + p3), fmaf(kLumaG, __ldg(rgb + p3 + HW), kLumaB * __ldg(rgb + p3 + 2 * HW)));
  }
}

// pass 1: ncc[j] = 0 (used; the value comes in pass 2) or kNccInvalid; counts[i] += used patches of pair i
__global__ void __launch_bounds__(256) k_ncc_valid(const __grid_constant__ BatchDev b,
                                                   const PairGeo* __restrict__ geo,
                                                   const unsigned* __restrict__ centers, long long n_per, int n_pairs,
                                                   const float* __restrict__ depth, const float* __restrict__ normal,
                                                   float* __restrict__ ncc, int* __restrict__ counts) {
  const long long n = n_per * n_pairs;
  for (long long j0 = blockIdx.x * (long long)blockDim.x; j0 < n; j0 += (long long)gridDim.x * blockDim.x) {
    const long long j = j0 + threadIdx.x;
    bool ok = false;
    int pair = 0;
    if (j < n) {
      pair = (int)(j / n_per);
      const ViewDev& vr = b.v[2 * pair + 1];
      const ViewDev& vs = b.v[2 * pair];
      Centre C;
      ok = centre_pos(vr, __ldg(centers + j), C);
      if (ok) {
        float d, nn[3];
        centre_fetch(vr, C, depth, normal, d, nn);
        ok = centre_plane(vr, d, nn, C);
      }
      if (ok) {
        const PairGeo g = geo[pair];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Warp w;
          warp_sample(vs, g, C, (k & 1) ? kHalf : -kHalf, (k & 2) ? kHalf : -kHalf, w);
          ok = ok && sample_ok(vs, w);
        }
      }
      ncc[j] = ok ? 0.f : kNccInvalid;
    }
    // one atomic per (warp, pair) present among the warp's used patches
    const unsigned lanes = __ballot_sync(0xffffffffu, ok);
    if (lanes) {
      const unsigned same = __match_any_sync(0xffffffffu, ok ? pair : -1);
      const unsigned mine = same & lanes;
      if (ok && (threadIdx.x & 31) == __ffs(mine) - 1) atomicAdd(counts + pair, __popc(mine));
    }
  }
}

// pass 2: one warp per patch; lane l holds samples l and l + 32 (l < 17)
__global__ void __launch_bounds__(256, 3) k_ncc_patch(const __grid_constant__ BatchDev b, NccArgs a,
                                                      const PairGeo* __restrict__ geo,
                                                      const unsigned* __restrict__ centers, long long n_per,
                                                      int n_pairs, const float* __restrict__ luma,
                                                      const float* __restrict__ depth,
                                                      const float* __restrict__ normal, const int* __restrict__ counts,
                                                      float* __restrict__ ncc, float* __restrict__ g_rgb,
                                                      float* __restrict__ g_depth, float* __restrict__ g_normal) {
  const int lane = threadIdx.x & 31;
  const long long n = n_per * n_pairs;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  const bool two = lane < kTaps - 32;
  // software pipeline over the warp's patches j, j + nw, ...: the flag and centre
  // of the next patch are loaded while this one samples, its D_hat and N_hat
  // while this one reduces, so the gathers overlap the current patch's work
  long long j = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  float flag = j < n ? ncc[j] : kNccInvalid;
  unsigned cidx = flag != kNccInvalid ? __ldg(centers + j) : 0u;
  Centre C{};
  float dn = 0.f, nn[3] = {0.f, 0.f, 0.f};
  if (flag != kNccInvalid) {
    const ViewDev& vr = b.v[2 * (int)(j / n_per) + 1];
    centre_pos(vr, cidx, C);
    centre_fetch(vr, C, depth, normal, dn, nn);
  }
  while (j < n) {
    const long long jn = j + nw;
    const float flag_n = jn < n ? ncc[jn] : kNccInvalid;
    const unsigned cidx_n = flag_n != kNccInvalid ? __ldg(centers + jn) : 0u;
    const bool used = flag != kNccInvalid;                    // warp-uniform
    const int pair = (int)(j / n_per);
    const ViewDev& vr = b.v[2 * pair + 1];
    const ViewDev& vs = b.v[2 * pair];
    float av[2] = {0.f, 0.f}, bv[2] = {0.f, 0.f}, gu[2] = {0.f, 0.f}, gv[2] = {0.f, 0.f};
    float da[2] = {0.f, 0.f}, db[2] = {0.f, 0.f};
    float saa = 1.f, sbb = 1.f, inv_den = 0.f, val = 0.f;
    Warp w[2];
    PairGeo g;
    if (used) {
      centre_plane(vr, dn, nn, C);                           // used: the pass-1 checks hold
      g = geo[pair];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int k = lane + 32 * s;
        if (s == 0 || two) {
          const int dy = k / kSide - kHalf, dx = k - (k / kSide) * kSide - kHalf;
          warp_sample(vs, g, C, dx, dy, w[s]);
          av[s] = __ldg(luma + C.p + (dy * vr.W + dx));
          bv[s] = luma_bilinear(vs, luma, w[s].u, w[s].v, gu[s], gv[s]);
        }
      }
      const float inv_n = 1.f / (float)kTaps;
      const float am = warp_sum(av[0] + av[1]) * inv_n, bm = warp_sum(bv[0] + bv[1]) * inv_n;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const bool on = s == 0 || two;
        da[s] = on ? av[s] - am : 0.f;
        db[s] = on ? bv[s] - bm : 0.f;
      }
      saa = warp_sum(fmaf(da[0], da[0], da[1] * da[1])) + a.eps;
      sbb = warp_sum(fmaf(db[0], db[0], db[1] * db[1])) + a.eps;
      const float sab = warp_sum(fmaf(da[0], db[0], da[1] * db[1]));
      inv_den = rsqrtf(saa * sbb);
      val = sab * inv_den;
      if (lane == 0) ncc[j] = val;
    }
    // the next patch's centre depth and normal
    Centre Cn = C;                                            // overwritten below for a used patch
    float dn_n = 0.f, nn_n[3] = {0.f, 0.f, 0.f};
    if (flag_n != kNccInvalid) {
      const ViewDev& vrn = b.v[2 * (int)(jn / n_per) + 1];
      centre_pos(vrn, cidx_n, Cn);
      centre_fetch(vrn, Cn, depth, normal, dn_n, nn_n);
    }
    if (used) {
      // dL/dNCC of this patch: L = lambda / (B/2) * mean over the pair's used patches of (1 - NCC)
      const float G = -a.lambda * rcp_approx((float)n_pairs * (float)__ldg(counts + pair));
      const float ca = G * inv_den, cb = G * val * rcp_approx(saa), cc = G * val * rcp_approx(sbb);
      const long long HWr = (long long)vr.W * vr.H;
      const long long c3 = 2 * vr.pix_off + C.p;
      float gm[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (!(s == 0 || two)) continue;
        const int k = lane + 32 * s;
        const int dy = k / kSide - kHalf, dx = k - (k / kSide) * kSide - kHalf;
        float* gq = g_rgb + c3 + (dy * vr.W + dx);
        const float ga = fmaf(ca, db[s], -cb * da[s]);        // dL/da_k
        atomicAdd(gq, kLumaR * ga);
        atomicAdd(gq + HWr, kLumaG * ga);
        atomicAdd(gq + 2 * HWr, kLumaB * ga);
        if (a.geometric) {
          const float gb = fmaf(ca, da[s], -cc * db[s]);      // dL/db_k
          const Warp& W = w[s];
          const float su = gb * gu[s] * vs.fx * W.iz, sv = gb * gv[s] * vs.fy * W.iz;
          // dL/dP = (su, sv, -(su P_x + sv P_y) / P_z); P depends on m through t (m . r_q)
          const float dPz = -(su * W.P[0] + sv * W.P[1]) * W.iz;
          const float sk = fmaf(su, g.t[0], fmaf(sv, g.t[1], dPz * g.t[2]));
          gm[0] = fmaf(sk, W.rq[0], gm[0]);
          gm[1] = fmaf(sk, W.rq[1], gm[1]);
          gm[2] += sk;
        }
      }
      if (a.geometric) {
        gm[0] = warp_sum(gm[0]);
        gm[1] = warp_sum(gm[1]);
        gm[2] = warp_sum(gm[2]);
        if (lane == 0) {
          // m = N / (D c), c = N . r_p
          const float idc = rcp_approx(C.d * C.c);
          const float gmm = fmaf(gm[0], C.m[0], fmaf(gm[1], C.m[1], gm[2] * C.m[2]));
          const float gmn = fmaf(gm[0], C.n[0], fmaf(gm[1], C.n[1], gm[2] * C.n[2]));
          atomicAdd(g_depth + C.p, -gmm * rcp_approx(C.d));
          const float k2 = gmn * idc * rcp_approx(C.c);
          atomicAdd(g_normal + c3, fmaf(gm[0], idc, -C.rp[0] * k2));
          atomicAdd(g_normal + c3 + HWr, fmaf(gm[1], idc, -C.rp[1] * k2));
          atomicAdd(g_normal + c3 + 2 * HWr, fmaf(gm[2], idc, -C.rp[2] * k2));
        }
      }
    }
    j = jn;
    flag = flag_n;
    C = Cn;
    dn = dn_n;
    nn[0] = nn_n[0];
    nn[1] = nn_n[1];
    nn[2] = nn_n[2];
  }
}

// pass 3: block (c, i) sums (1 - NCC) over chunk c of pair i's patches in a fixed
// order; the last block to finish adds the chunks, then the pairs' means, in order
__global__ void __launch_bounds__(256) k_ncc_final(const float* __restrict__ ncc, long long n_per, int n_pairs,
                                                   int* __restrict__ counts, float* __restrict__ partial,
                                                   float lambda, float* __restrict__ loss) {
  __shared__ float red[256];
  __shared__ bool last;
  const int c = blockIdx.x, i = blockIdx.y;
  const long long chunk = (n_per + kNccChunks - 1) / kNccChunks;
  const long long k0 = c * chunk, k1 = min(n_per, k0 + chunk);
  const float* q = ncc + (long long)i * n_per;
  float acc = 0.f;
#pragma unroll 4
  for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const float v = __ldg(q + k);
    acc += v != kNccInvalid ? 1.f - v : 0.f;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[i * kNccChunks + c] = red[0];
    __threadfence();
    last = atomicAdd(counts + kNccDone, 1) == n_pairs * kNccChunks - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    float total = 0.f;
    for (int p = 0; p < n_pairs; ++p) {
      float sum = 0.f;
      for (int k = 0; k < kNccChunks; ++k) sum += *(volatile float*)(partial + p * kNccChunks + k);
      const int cnt = *(volatile int*)(counts + p);
      if (cnt > 0) total += sum / (float)cnt;
    }
    const float L = total / (float)n_pairs;
    loss[0] = lambda * L;
    loss[1] = L;
  }
}

cudaError_t launch_ncc(const BatchDev& b, const NccArgs& a, const unsigned* centers, long long n_per, int n_pairs,
                       const float* rgb, const float* depth, const float* normal, float* ncc, float* loss,
                       float* g_rgb, float* g_depth, float* g_normal, void* scratch, float* luma, int num_sms,
                       cudaStream_t st) {
  int* counts = reinterpret_cast<int*>(scratch);
  float* partial = reinterpret_cast<float*>(counts + kNccDone + 1);
  PairGeo* geo = reinterpret_cast<PairGeo*>(partial + kMaxViews / 2 * kNccChunks);
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (kNccDone + 1), st);
  if (e != cudaSuccess) return e;
  const long long n = n_per * n_pairs;
  if (n_pairs == 0 || n == 0) return cudaMemsetAsync(loss, 0, 2 * sizeof(float), st);
  const long long n_pix = b.v[2 * n_pairs - 1].pix_off + (long long)b.v[2 * n_pairs - 1].W * b.v[2 * n_pairs - 1].H;
  bool quad = (reinterpret_cast<uintptr_t>(rgb) & 15) == 0 && (reinterpret_cast<uintptr_t>(luma) & 15) == 0;
  for (int v = 0; v < 2 * n_pairs; ++v)
    quad = quad && (b.v[v].pix_off % 4 == 0) && (((long long)b.v[v].W * b.v[v].H) % 4 == 0);
  const long long blk0 = std::min<long long>((n_pix / (quad ? 4 : 1) + 255) / 256, (long long)num_sms * 16);
  k_ncc_luma<<<(unsigned)std::max<long long>(blk0, 1), 256, 0, st>>>(b, n_pairs, rgb, n_pix, quad, luma, geo);
  const long long blk1 = std::min<long long>((n + 255) / 256, (long long)num_sms * 8);
  k_ncc_valid<<<(unsigned)blk1, 256, 0, st>>>(b, geo, centers, n_per, n_pairs, depth, normal, ncc, counts);
  const long long blk2 = std::min<long long>((n + 7) / 8, (long long)num_sms * 32);
  k_ncc_patch<<<(unsigned)blk2, 256, 0, st>>>(b, a, geo, centers, n_per, n_pairs, luma, depth, normal, counts, ncc,
                                              g_rgb, g_depth, g_normal);
  k_ncc_final<<<dim3(kNccChunks, n_pairs), 256, 0, st>>>(ncc, n_per, n_pairs, counts, partial, a.lambda, loss);
  return cudaGetLastError();
}

size_t ncc_scratch_bytes() {
  return sizeof(int) * (kNccDone + 1) + sizeof(float) * (kMaxViews / 2) * kNccChunks +
         sizeof(PairGeo) * (kMaxViews / 2) + 64;
}

}  // namespace pgs
