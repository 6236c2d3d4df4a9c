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
// Three kernels: validity and per-pair counts (one thread per patch; integer
// atomics, so the counts are exact), the patch pass (one warp per valid patch:
// NCC, gradients scaled by the now known 1 / count, float atomics into the
// image gradients), and a one-block fixed-order reduction of the loss.
#include <algorithm>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

namespace {

constexpr int kHalf = 3, kSide = 7, kTaps = kSide * kSide;
constexpr float kLumaR = 0.299f, kLumaG = 0.587f, kLumaB = 0.114f;

// relative pose of the pair: X_s = R X_r + t
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
  float d, n[3], rp[3], c, m[3];
};

__device__ __forceinline__ bool load_centre(const ViewDev& vr, unsigned cidx, const float* __restrict__ depth,
                                            const float* __restrict__ normal, Centre& C) {
  const long long HW = (long long)vr.W * vr.H;
  if ((long long)cidx >= HW) return false;
  C.y = (int)(cidx / (unsigned)vr.W);
  C.x = (int)(cidx - (unsigned)C.y * (unsigned)vr.W);
  if (C.x < kHalf || C.y < kHalf || C.x > vr.W - 1 - kHalf || C.y > vr.H - 1 - kHalf) return false;
  C.p = vr.pix_off + cidx;
  C.d = __ldg(depth + C.p);
  const long long p3 = 3 * vr.pix_off + cidx;
  C.n[0] = __ldg(normal + p3);
  C.n[1] = __ldg(normal + p3 + HW);
  C.n[2] = __ldg(normal + p3 + 2 * HW);
  C.rp[0] = ((float)C.x + 0.5f - vr.cx) / vr.fx;
  C.rp[1] = ((float)C.y + 0.5f - vr.cy) / vr.fy;
  C.rp[2] = 1.f;
  C.c = fmaf(C.n[0], C.rp[0], fmaf(C.n[1], C.rp[1], C.n[2]));
  if (!(C.d > 0.f) || !(fabsf(C.c) >= 1e-8f)) return false;
  const float den = C.d * C.c;
  C.m[0] = C.n[0] / den;
  C.m[1] = C.n[1] / den;
  C.m[2] = C.n[2] / den;
  return true;
}

// warped position of patch sample k (row-major over dy, dx in [-3, 3]);
// rq: the reference ray of the sample, P: partner camera coordinates up to the
// positive factor m . r_q
struct Warp {
  float rq[3], mr, P[3], u, v;
};

__device__ __forceinline__ void warp_sample(const ViewDev& vr, const ViewDev& vs, const PairGeo& g, const Centre& C,
                                            int k, Warp& w) {
  const int dy = k / kSide - kHalf, dx = k - (k / kSide) * kSide - kHalf;
  w.rq[0] = ((float)(C.x + dx) + 0.5f - vr.cx) / vr.fx;
  w.rq[1] = ((float)(C.y + dy) + 0.5f - vr.cy) / vr.fy;
  w.rq[2] = 1.f;
  w.mr = fmaf(C.m[0], w.rq[0], fmaf(C.m[1], w.rq[1], C.m[2]));
#pragma unroll
  for (int i = 0; i < 3; ++i)
    w.P[i] = fmaf(g.t[i], w.mr, fmaf(g.R[3 * i + 0], w.rq[0], fmaf(g.R[3 * i + 1], w.rq[1], g.R[3 * i + 2])));
  w.u = fmaf(vs.fx, w.P[0] / w.P[2], vs.cx);
  w.v = fmaf(vs.fy, w.P[1] / w.P[2], vs.cy);
}

// the sample has the plane in front of both cameras and its bilinear footprint
// (pixel centres at +1/2) inside the partner frame
__device__ __forceinline__ bool sample_ok(const ViewDev& vs, const Warp& w) {
  if (!(w.mr > 0.f && w.P[2] > 0.f)) return false;
  const float fu = floorf(w.u - 0.5f), fv = floorf(w.v - 0.5f);
  return fu >= 0.f && fv >= 0.f && fu + 1.f <= (float)(vs.W - 1) && fv + 1.f <= (float)(vs.H - 1);
}

__device__ __forceinline__ float luma_at(const float* __restrict__ rgb, long long p3, long long HW) {
  return fmaf(kLumaR, __ldg(rgb + p3), fmaf(kLumaG, __ldg(rgb + p3 + HW), kLumaB * __ldg(rgb + p3 + 2 * HW)));
}

// partner luma, bilinear at (u, v), and its slope (du, dv); indices clamped so
// that the reads stay inside the view even if the validity pass and this one
// round a position differently
__device__ __forceinline__ float luma_bilinear(const ViewDev& vs, const float* __restrict__ rgb, float u, float v,
                                               float& gu, float& gv) {
  const float x = u - 0.5f, y = v - 0.5f;
  const float fx = floorf(x), fy = floorf(y);
  const int i0 = min(max((int)fx, 0), vs.W - 2), j0 = min(max((int)fy, 0), vs.H - 2);
  const float ax = x - fx, ay = y - fy;
  const long long HW = (long long)vs.W * vs.H;
  const long long p3 = 3 * vs.pix_off + (long long)j0 * vs.W + i0;
  const float g00 = luma_at(rgb, p3, HW), g10 = luma_at(rgb, p3 + 1, HW);
  const float g01 = luma_at(rgb, p3 + vs.W, HW), g11 = luma_at(rgb, p3 + vs.W + 1, HW);
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

// pass 1: ncc[j] = 0 (valid, value filled by pass 2) or kNccInvalid; counts[i] += valid patches of pair i
__global__ void __launch_bounds__(256) k_ncc_valid(const __grid_constant__ BatchDev b, const unsigned* __restrict__ centers,
                                                   long long n_per, int n_pairs, const float* __restrict__ depth,
                                                   const float* __restrict__ normal, float* __restrict__ ncc,
                                                   int* __restrict__ counts) {
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
      ok = load_centre(vr, __ldg(centers + j), depth, normal, C);
      if (ok) {
        PairGeo g;
        pair_geo(vr, vs, g);
#pragma unroll 1
        for (int k = 0; k < kTaps && ok; ++k) {
          Warp w;
          warp_sample(vr, vs, g, C, k, w);
          ok = sample_ok(vs, w);
        }
      }
      ncc[j] = ok ? 0.f : kNccInvalid;
    }
    // one atomic per (warp, pair) present among the warp's valid patches
    const unsigned lanes = __ballot_sync(0xffffffffu, ok);
    if (lanes) {
      const unsigned same = __match_any_sync(0xffffffffu, ok ? pair : -1);
      const unsigned mine = same & lanes;
      if (ok && (threadIdx.x & 31) == __ffs(mine) - 1) atomicAdd(counts + pair, __popc(mine));
    }
  }
}

// pass 2: one warp per patch; lane l holds samples l and l + 32 (l < 17)
__global__ void __launch_bounds__(256) k_ncc_patch(const __grid_constant__ BatchDev b, NccArgs a,
                                                   const unsigned* __restrict__ centers, long long n_per, int n_pairs,
                                                   const float* __restrict__ rgb, const float* __restrict__ depth,
                                                   const float* __restrict__ normal, const int* __restrict__ counts,
                                                   float* __restrict__ ncc, float* __restrict__ g_rgb,
                                                   float* __restrict__ g_depth, float* __restrict__ g_normal) {
  const int lane = threadIdx.x & 31;
  const long long n = n_per * n_pairs;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long j = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += nw) {
    if (ncc[j] == kNccInvalid) continue;                     // warp-uniform
    const int pair = (int)(j / n_per);
    const ViewDev& vr = b.v[2 * pair + 1];
    const ViewDev& vs = b.v[2 * pair];
    Centre C;
    load_centre(vr, __ldg(centers + j), depth, normal, C);   // valid: the pass-1 checks hold
    PairGeo g;
    pair_geo(vr, vs, g);
    const long long HWr = (long long)vr.W * vr.H;
    const bool two = lane < kTaps - 32;
    float av[2], bv[2], gu[2], gv[2];
    Warp w[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int k = lane + 32 * s;
      av[s] = bv[s] = gu[s] = gv[s] = 0.f;
      if (s == 0 || two) {
        warp_sample(vr, vs, g, C, k, w[s]);
        const int dy = k / kSide - kHalf, dx = k - (k / kSide) * kSide - kHalf;
        const long long q3 = 3 * vr.pix_off + (long long)(C.y + dy) * vr.W + (C.x + dx);
        av[s] = luma_at(rgb, q3, HWr);
        bv[s] = luma_bilinear(vs, rgb, w[s].u, w[s].v, gu[s], gv[s]);
      }
    }
    const float inv_n = 1.f / (float)kTaps;
    const float am = warp_sum(av[0] + av[1]) * inv_n, bm = warp_sum(bv[0] + bv[1]) * inv_n;
    float da[2], db[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const bool on = s == 0 || two;
      da[s] = on ? av[s] - am : 0.f;
      db[s] = on ? bv[s] - bm : 0.f;
    }
    const float saa = warp_sum(fmaf(da[0], da[0], da[1] * da[1])) + a.eps;
    const float sbb = warp_sum(fmaf(db[0], db[0], db[1] * db[1])) + a.eps;
    const float sab = warp_sum(fmaf(da[0], db[0], da[1] * db[1]));
    const float inv_den = 1.f / sqrtf(saa * sbb);
    const float val = sab * inv_den;
    if (lane == 0) ncc[j] = val;
    // dL/dNCC of this patch: L = lambda / (B/2) * mean over the pair's valid patches of (1 - NCC)
    const float G = -a.lambda / ((float)n_pairs * (float)__ldg(counts + pair));
    float gm[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (!(s == 0 || two)) continue;
      const int k = lane + 32 * s;
      const int dy = k / kSide - kHalf, dx = k - (k / kSide) * kSide - kHalf;
      const long long q3 = 3 * vr.pix_off + (long long)(C.y + dy) * vr.W + (C.x + dx);
      const float ga = G * (db[s] * inv_den - val * da[s] / saa);     // dL/da_k
      atomicAdd(g_rgb + q3, kLumaR * ga);
      atomicAdd(g_rgb + q3 + HWr, kLumaG * ga);
      atomicAdd(g_rgb + q3 + 2 * HWr, kLumaB * ga);
      if (a.geometric) {
        const float gb = G * (da[s] * inv_den - val * db[s] / sbb);   // dL/db_k
        const Warp& W = w[s];
        const float iz = 1.f / W.P[2];
        const float su = gb * gu[s] * vs.fx * iz, sv = gb * gv[s] * vs.fy * iz;
        // dL/dP = (su, sv, -(su P_x + sv P_y) / P_z); P depends on m through t (m . r_q)
        const float dPz = -(su * W.P[0] + sv * W.P[1]) * iz;
        const float sk = fmaf(su, g.t[0], fmaf(sv, g.t[1], dPz * g.t[2]));
        gm[0] = fmaf(sk, W.rq[0], gm[0]);
        gm[1] = fmaf(sk, W.rq[1], gm[1]);
        gm[2] = fmaf(sk, W.rq[2], gm[2]);
      }
    }
    if (a.geometric) {
      gm[0] = warp_sum(gm[0]);
      gm[1] = warp_sum(gm[1]);
      gm[2] = warp_sum(gm[2]);
      if (lane == 0) {
        // m = N / (D c), c = N . r_p
        const float dc = C.d * C.c;
        const float gmm = fmaf(gm[0], C.m[0], fmaf(gm[1], C.m[1], gm[2] * C.m[2]));
        const float gmn = fmaf(gm[0], C.n[0], fmaf(gm[1], C.n[1], gm[2] * C.n[2]));
        atomicAdd(g_depth + C.p, -gmm / C.d);
        const long long p3 = 3 * vr.pix_off + (C.p - vr.pix_off);
        const float k2 = gmn / (dc * C.c);
        atomicAdd(g_normal + p3, gm[0] / dc - C.rp[0] * k2);
        atomicAdd(g_normal + p3 + HWr, gm[1] / dc - C.rp[1] * k2);
        atomicAdd(g_normal + p3 + 2 * HWr, gm[2] / dc - C.rp[2] * k2);
      }
    }
  }
}

// pass 3: one block; per pair the fixed-order sum of (1 - NCC) over valid patches
__global__ void __launch_bounds__(1024) k_ncc_final(const float* __restrict__ ncc, long long n_per, int n_pairs,
                                                    const int* __restrict__ counts, float lambda,
                                                    float* __restrict__ loss) {
  __shared__ float red[1024];
  float total = 0.f;
  for (int i = 0; i < n_pairs; ++i) {
    float acc = 0.f;
    for (long long k = threadIdx.x; k < n_per; k += blockDim.x) {
      const float v = ncc[(long long)i * n_per + k];
      if (v != kNccInvalid) acc += 1.f - v;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    const int cnt = counts[i];
    if (cnt > 0) total += red[0] / (float)cnt;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float L = n_pairs > 0 ? total / (float)n_pairs : 0.f;
    loss[0] = lambda * L;
    loss[1] = L;
  }
}

void launch_ncc(const BatchDev& b, const NccArgs& a, const unsigned* centers, long long n_per, int n_pairs,
                const float* rgb, const float* depth, const float* normal, float* ncc, float* loss, float* g_rgb,
                float* g_depth, float* g_normal, int* counts, int num_sms, cudaStream_t st) {
  cudaMemsetAsync(counts, 0, sizeof(int) * kMaxViews / 2, st);
  const long long n = n_per * n_pairs;
  if (n > 0) {
    const long long blk1 = std::min<long long>((n + 255) / 256, (long long)num_sms * 8);
    k_ncc_valid<<<(unsigned)blk1, 256, 0, st>>>(b, centers, n_per, n_pairs, depth, normal, ncc, counts);
    const long long blk2 = std::min<long long>((n + 7) / 8, (long long)num_sms * 16);
    k_ncc_patch<<<(unsigned)blk2, 256, 0, st>>>(b, a, centers, n_per, n_pairs, rgb, depth, normal, counts, ncc,
                                                g_rgb, g_depth, g_normal);
  }
  k_ncc_final<<<1, 1024, 0, st>>>(ncc, n_per, n_pairs, counts, a.lambda, loss);
}

}  // namespace pgs
