// Anchor LoD/frustum cull, shared-decoder forward (FP32 SIMT form), EWA
// projection and tile counting.
//
// Decoder (Eq. 4): X = [F_v, (x_v - o_c)/|x_v - o_c|]; H = ReLU(W1 X + b1);
// Z = W2 H + b2 blocked [opacity x10 | colour x30 | scale x30 | quat x40];
// opacity = sigmoid, colour = sigmoid, scale = l_v * sigmoid, quat = normalise;
// mu_j = x_v + O_j * l_v with l_v = exp(log_l).
// Projection: EWA splatting (3DGS) with J clamped at jclamp * tan(fov/2) and a
// dilation added to the 2D covariance; normal = rotation axis of the smallest
// scale turned to face the camera, in the camera frame (Eq. 6); plane distance
// d = n . mu_c (Eq. 7).
#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

// Project one 3D Gaussian into view v: writes the 64 B record, its tile count
// and its depth key (0xffffffff when it touches no tile).  mu_lo (optional) is
// the low part of a double-float mean: the camera-frame mean, hence the FP32
// depth key and the 2D mean, come out correctly rounded.
__device__ void project_gaussian(const BatchDev& b, const ViewDev& v, const float mu[3], const float s[3],
                                 const float q[4], float opacity, const float col[3], float4* rec,
                                 uint32_t* count_out, uint32_t* key_out, const float* mu_lo = nullptr) {
  const ParamsDev& p = b.p;
  float xh, xl, yh, yl, zh, zl;
  float ex = 0.f, ey = 0.f, ez = 0.f;
  if (mu_lo) {
    ex = v.R[0] * mu_lo[0] + v.R[1] * mu_lo[1] + v.R[2] * mu_lo[2];
    ey = v.R[3] * mu_lo[0] + v.R[4] * mu_lo[1] + v.R[5] * mu_lo[2];
    ez = v.R[6] * mu_lo[0] + v.R[7] * mu_lo[1] + v.R[8] * mu_lo[2];
  }
  dot3_add(&v.R[0], mu[0], mu[1], mu[2], v.t[0], xh, xl, ex);
  dot3_add(&v.R[3], mu[0], mu[1], mu[2], v.t[1], yh, yl, ey);
  dot3_add(&v.R[6], mu[0], mu[1], mu[2], v.t[2], zh, zl, ez);
  const float x = xh, y = yh, z = zh;
  bool valid = (z >= p.near_plane) && (opacity >= p.alpha_min);
  const float iz = 1.f / z;
  const float txz = fminf(fmaxf(x * iz, -v.lim_x), v.lim_x);
  const float tyz = fminf(fmaxf(y * iz, -v.lim_y), v.lim_y);
  const float J00 = v.fx * iz, J02 = -v.fx * txz * iz;
  const float J11 = v.fy * iz, J12 = -v.fy * tyz * iz;
  float Rg[9];
  quat_to_rot(q[0], q[1], q[2], q[3], Rg);
  // T = J W (2x3)
  float T0[3], T1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T0[c] = J00 * v.R[c] + J02 * v.R[6 + c];
    T1[c] = J11 * v.R[3 + c] + J12 * v.R[6 + c];
  }
  // U = T Rg S ; cov = U U^T
  float a = 0.f, bb = 0.f, c = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float u0 = (T0[0] * Rg[k] + T0[1] * Rg[3 + k] + T0[2] * Rg[6 + k]) * s[k];
    float u1 = (T1[0] * Rg[k] + T1[1] * Rg[3 + k] + T1[2] * Rg[6 + k]) * s[k];
    a += u0 * u0;
    bb += u0 * u1;
    c += u1 * u1;
  }
  a += p.dilation;
  c += p.dilation;
  const float det = a * c - bb * bb;
  valid = valid && (det > 0.f);
  const float idet = 1.f / det;
  float mxh, mxl, myh, myl;
  df_scaled_ratio(v.fx, xh, xl, zh, zl, mxh, mxl);
  df_scaled_ratio(v.fy, yh, yl, zh, zl, myh, myl);
  // normal: column of the smallest scale (first on ties), camera frame, facing the camera
  int k = 0;
  if (s[1] < s[k]) k = 1;
  if (s[2] < s[k]) k = 2;
  float nw0 = Rg[k], nw1 = Rg[3 + k], nw2 = Rg[6 + k];
  float n0 = v.R[0] * nw0 + v.R[1] * nw1 + v.R[2] * nw2;
  float n1 = v.R[3] * nw0 + v.R[4] * nw1 + v.R[5] * nw2;
  float n2 = v.R[6] * nw0 + v.R[7] * nw1 + v.R[8] * nw2;
  float facing = n0 * x + n1 * y + n2 * z;
  if (facing > 0.f) { n0 = -n0; n1 = -n1; n2 = -n2; }
  const float d = n0 * x + n1 * y + n2 * z;
  float4 r0 = make_float4(mxh, myh, mxl, myl);
  float4 r1 = make_float4(c * idet, -bb * idet, a * idet, opacity);
  float4 r2 = make_float4(col[0], col[1], col[2], d);
  float4 r3 = make_float4(n0, n1, n2, z);
  valid = valid && isfinite(mxh) && isfinite(myh) && isfinite(r1.x) && isfinite(r1.y) && isfinite(r1.z) &&
          isfinite(d) && isfinite(n0) && isfinite(n1) && isfinite(n2) && isfinite(col[0]) &&
          isfinite(col[1]) && isfinite(col[2]);
  uint32_t cnt = 0;
  if (valid) {
    TileEllipse e;
    if (tile_ellipse_setup(r0, r1, p, e)) {
      for_each_tile_row(e, v, p.tile_w, p.tile_h, [&](int, int c0, int c1) { cnt += (uint32_t)(c1 - c0 + 1); });
    }
  }
  rec[0] = r0;
  rec[1] = r1;
  rec[2] = r2;
  rec[3] = r3;
  *count_out = cnt;
  *key_out = cnt ? __float_as_uint(z) : 0xffffffffu;
}

// ---------------------------------------------------------------- explicit Gaussians
__global__ void __launch_bounds__(256) k_project_explicit(const __grid_constant__ BatchDev b,
                                                          pgs_explicit_ptrs P, long long N, float4* __restrict__ rec,
                                                          uint32_t* __restrict__ counts,
                                                          uint32_t* __restrict__ keys) {
  const long long G = N * b.n_views;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G;
       g += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(g / N);
    const long long i = g - (long long)v * N;
    float mu[3] = {P.means[3 * i], P.means[3 * i + 1], P.means[3 * i + 2]};
    float s[3] = {expf(P.log_scales[3 * i]), expf(P.log_scales[3 * i + 1]), expf(P.log_scales[3 * i + 2])};
    float q[4] = {P.quats[4 * i], P.quats[4 * i + 1], P.quats[4 * i + 2], P.quats[4 * i + 3]};
    float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (qn < 1e-12f) { q[0] = 1.f; q[1] = q[2] = q[3] = 0.f; }
    else { float iq = 1.f / qn; q[0] *= iq; q[1] *= iq; q[2] *= iq; q[3] *= iq; }
    float op = sigmoidf_(P.opacity_logits[i]);
    float col[3] = {P.colors[3 * i], P.colors[3 * i + 1], P.colors[3 * i + 2]};
    project_gaussian(b, b.v[v], mu, s, q, op, col, rec + g * kRecF4, counts + g, keys + g);
  }
}

// ---------------------------------------------------------------- anchors: cull
// Level rule (Sec. 3.1, Octree-GS): level <= clamp(floor(log2(d0 / d)), 0, K-1),
// written as comparisons with the exact thresholds d0 / 2^m.  Frustum rule:
// a conservative bounding sphere of the anchor's 10 Gaussians (radius
// max(l) (max_j |O_j| + 3.4), i.e. past the alpha = 1/255 level of any
// Gaussian with scale <= l) whose screen bound (twice the projected radius
// + 4 px) misses the image, or which lies wholly behind the near plane.
__global__ void __launch_bounds__(256) k_anchor_cull(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A,
                                                     long long Na, uint32_t* __restrict__ flags) {
  const long long total = Na * b.n_views;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int vi = (int)(idx / Na);
    const long long i = idx - (long long)vi * Na;
    const ViewDev& v = b.v[vi];
    const float x0 = A.x[3 * i], x1 = A.x[3 * i + 1], x2 = A.x[3 * i + 2];
    const float dx = x0 - v.center[0], dy = x1 - v.center[1], dz = x2 - v.center[2];
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    int L = 0;
    for (int m = 1; m < b.p.n_levels; ++m) L += (dist <= b.p.lod_d0 / (float)(1 << m)) ? 1 : 0;
    const int level = A.level[i];
    bool keep = level >= 0 && level <= L;
    if (keep) {
      float lm = fmaxf(fmaxf(A.log_l[3 * i], A.log_l[3 * i + 1]), A.log_l[3 * i + 2]);
      lm = expf(lm);
      float om = 0.f;
      for (int j = 0; j < kNOff; ++j) {
        const float* o = A.offsets + (i * kNOff + j) * 3;
        om = fmaxf(om, sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]));
      }
      const float Rs = lm * (om + 3.4f);
      const float xc = v.R[0] * x0 + v.R[1] * x1 + v.R[2] * x2 + v.t[0];
      const float yc = v.R[3] * x0 + v.R[4] * x1 + v.R[5] * x2 + v.t[1];
      const float zc = v.R[6] * x0 + v.R[7] * x1 + v.R[8] * x2 + v.t[2];
      if (zc + Rs < b.p.near_plane) {
        keep = false;
      } else if (zc - Rs > b.p.near_plane) {
        const float rho = fmaxf(v.fx, v.fy) * Rs / sqrtf(zc * zc - Rs * Rs);
        const float u = v.fx * xc / zc + v.cx, w = v.fy * yc / zc + v.cy;
        const float m = 2.f * rho + 4.f;
        if (u + m < 0.f || u - m > (float)v.W || w + m < 0.f || w - m > (float)v.H) keep = false;
      }
      if (!isfinite(Rs) || !isfinite(zc)) keep = false;
    }
    flags[idx] = keep ? 1u : 0u;
  }
}

__global__ void k_compact_rows(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ offs,
                               long long total, long long Na, uint32_t* __restrict__ rows, long long cap,
                               uint32_t* err) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    if (!flags[idx]) continue;
    const long long o = offs[idx];
    if (o >= cap) { set_flag(err, kFlagCapacity); continue; }
    const int vi = (int)(idx / Na);
    const long long i = idx - (long long)vi * Na;
    rows[o] = ((uint32_t)vi << 27) | (uint32_t)i;
  }
}

// ---------------------------------------------------------------- anchors: decode + project (FP32)
struct MlpSmem {
  float W1[kHidden][kMaxIn];
  float b1[kHidden];
  float W2[kOut][kHidden];
  float b2[kOut];
};

__device__ __forceinline__ void load_mlp_smem(MlpSmem& m, const pgs_mlp_ptrs& w, int in_dim) {
  for (int t = threadIdx.x; t < kHidden * in_dim; t += blockDim.x) m.W1[t / in_dim][t % in_dim] = w.W1[t];
  for (int t = threadIdx.x; t < kHidden; t += blockDim.x) m.b1[t] = w.b1[t];
  for (int t = threadIdx.x; t < kOut * kHidden; t += blockDim.x) m.W2[t / kHidden][t % kHidden] = w.W2[t];
  for (int t = threadIdx.x; t < kOut; t += blockDim.x) m.b2[t] = w.b2[t];
}

// decoder input of one (view, anchor) row; returns |x - o_c|
__device__ __forceinline__ float decoder_input(const pgs_anchor_ptrs& A, const ViewDev& v, long long a, int in_dim,
                                               float* X) {
  const float dx = A.x[3 * a] - v.center[0], dy = A.x[3 * a + 1] - v.center[1], dz = A.x[3 * a + 2] - v.center[2];
  const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
  const float id = 1.f / dist;
  const float4* F4 = reinterpret_cast<const float4*>(A.feat + a * kFeat);
#pragma unroll
  for (int j = 0; j < kFeat / 4; ++j) {
    float4 f = F4[j];
    X[4 * j] = f.x; X[4 * j + 1] = f.y; X[4 * j + 2] = f.z; X[4 * j + 3] = f.w;
  }
  X[32] = dx * id; X[33] = dy * id; X[34] = dz * id;
  if (in_dim == 36) X[35] = dist;
  return dist;
}

__global__ void __launch_bounds__(256) k_decode_project(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A,
                                                        pgs_mlp_ptrs Wt, const uint32_t* __restrict__ rows,
                                                        const long long* __restrict__ n_rows_p, long long cap,
                                                        float4* __restrict__ rec, uint32_t* __restrict__ counts,
                                                        uint32_t* __restrict__ keys, DecodeOut dec) {
  __shared__ MlpSmem m;
  const int in_dim = b.p.in_dim;
  load_mlp_smem(m, Wt, in_dim);
  __syncthreads();
  const long long n_rows = min(*n_rows_p, cap);
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n_rows;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t rw = rows[r];
    const int vi = rw >> 27;
    const long long a = rw & ((1u << 27) - 1);
    const ViewDev& v = b.v[vi];
    float X[kMaxIn];
    decoder_input(A, v, a, in_dim, X);
    float H[kHidden];
#pragma unroll 4
    for (int i = 0; i < kHidden; ++i) {
      float acc = m.b1[i];
      for (int j = 0; j < in_dim; ++j) acc = fmaf(m.W1[i][j], X[j], acc);
      H[i] = fmaxf(acc, 0.f);
    }
    const float l[3] = {expf(A.log_l[3 * a]), expf(A.log_l[3 * a + 1]), expf(A.log_l[3 * a + 2])};
    const float xa[3] = {A.x[3 * a], A.x[3 * a + 1], A.x[3 * a + 2]};
#pragma unroll 1
    for (int j = 0; j < kNOff; ++j) {
      float z[11];
      const int idx[11] = {j, 10 + 3 * j, 11 + 3 * j, 12 + 3 * j, 40 + 3 * j, 41 + 3 * j, 42 + 3 * j,
                           70 + 4 * j, 71 + 4 * j, 72 + 4 * j, 73 + 4 * j};
#pragma unroll
      for (int t = 0; t < 11; ++t) {
        float acc = m.b2[idx[t]];
#pragma unroll
        for (int h = 0; h < kHidden; ++h) acc = fmaf(m.W2[idx[t]][h], H[h], acc);
        z[t] = acc;
      }
      const float op = sigmoidf_(z[0]);
      const float col[3] = {sigmoidf_(z[1]), sigmoidf_(z[2]), sigmoidf_(z[3])};
      const float s[3] = {l[0] * sigmoidf_(z[4]), l[1] * sigmoidf_(z[5]), l[2] * sigmoidf_(z[6])};
      float q[4] = {z[7], z[8], z[9], z[10]};
      const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      if (qn < 1e-12f) { q[0] = 1.f; q[1] = q[2] = q[3] = 0.f; }
      else { const float iq = 1.f / qn; q[0] *= iq; q[1] *= iq; q[2] *= iq; q[3] *= iq; }
      const float* O = A.offsets + (a * kNOff + j) * 3;
      // mu = x + O * l as a double-float (TwoProduct + TwoSum)
      float mu[3], mu_lo[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float pr = __fmul_rn(O[k], l[k]);
        const float e1 = __fmaf_rn(O[k], l[k], -pr);
        float e2;
        two_sum(xa[k], pr, mu[k], e2);
        mu_lo[k] = __fadd_rn(e1, e2);
      }
      const long long g = r * kNOff + j;
      if (dec.mu) {  // decoded Gaussians for pgs_decode_anchors
        dec.mu[3 * g] = mu[0]; dec.mu[3 * g + 1] = mu[1]; dec.mu[3 * g + 2] = mu[2];
        dec.opacity[g] = op;
        dec.color[3 * g] = col[0]; dec.color[3 * g + 1] = col[1]; dec.color[3 * g + 2] = col[2];
        dec.scale[3 * g] = s[0]; dec.scale[3 * g + 1] = s[1]; dec.scale[3 * g + 2] = s[2];
        dec.quat[4 * g] = q[0]; dec.quat[4 * g + 1] = q[1]; dec.quat[4 * g + 2] = q[2]; dec.quat[4 * g + 3] = q[3];
      }
      if (rec) project_gaussian(b, v, mu, s, q, op, col, rec + g * kRecF4, counts + g, keys + g, mu_lo);
    }
  }
}

}  // namespace pgs
