// EWA projection of one Gaussian and the decoder's per-Gaussian epilogue,
// shared by the FP32 and the tensor-core decoder kernels.
#pragma once
#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

// Project one 3D Gaussian into view v: writes the 64 B record, its tile count
// and its depth key (0xffffffff when it touches no tile).  mu_lo (optional) is
// the low part of a double-float mean: the camera-frame mean, hence the FP32
// depth key and the 2D mean, come out correctly rounded.  A non-finite mean,
// scale, rotation, opacity or colour raises kFlagNonfinite in *err (if given);
// such a Gaussian is never drawn.
__device__ __forceinline__ void project_gaussian(const BatchDev& b, const ViewDev& v, const float mu[3], const float s[3],
                                 const float q[4], float opacity, const float col[3], float4* rec,
                                 uint32_t* count_out, uint32_t* key_out, uint32_t* err,
                                 const float* mu_lo = nullptr) {
  const ParamsDev& p = b.p;
  if (err && !(isfinite(mu[0]) && isfinite(mu[1]) && isfinite(mu[2]) && isfinite(s[0]) && isfinite(s[1]) &&
               isfinite(s[2]) && isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]) &&
               isfinite(opacity) && isfinite(col[0]) && isfinite(col[1]) && isfinite(col[2])))
    set_flag(err, kFlagNonfinite);
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

// Decoder epilogue for Gaussian j of an anchor (Eq. 4): z = its 11 outputs
// (opacity, colour x3, scale x3, quaternion x4) before activation.
__device__ __forceinline__ void decode_gaussian(const BatchDev& b, const ViewDev& v, const float z[11], const float l[3],
                                                const float xa[3], const float* O, long long g, float4* rec,
                                                uint32_t* counts, uint32_t* keys, const DecodeOut& dec,
                                                uint32_t* err) {
  const float op = sigmoidf_(z[0]);
  const float col[3] = {sigmoidf_(z[1]), sigmoidf_(z[2]), sigmoidf_(z[3])};
  const float s[3] = {l[0] * sigmoidf_(z[4]), l[1] * sigmoidf_(z[5]), l[2] * sigmoidf_(z[6])};
  float q[4] = {z[7], z[8], z[9], z[10]};
  const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (qn < 1e-12f) { q[0] = 1.f; q[1] = q[2] = q[3] = 0.f; }
  else { const float iq = 1.f / qn; q[0] *= iq; q[1] *= iq; q[2] *= iq; q[3] *= iq; }
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
  if (dec.mu) {  // decoded Gaussians for pgs_decode_anchors
    dec.mu[3 * g] = mu[0]; dec.mu[3 * g + 1] = mu[1]; dec.mu[3 * g + 2] = mu[2];
    dec.opacity[g] = op;
    dec.color[3 * g] = col[0]; dec.color[3 * g + 1] = col[1]; dec.color[3 * g + 2] = col[2];
    dec.scale[3 * g] = s[0]; dec.scale[3 * g + 1] = s[1]; dec.scale[3 * g + 2] = s[2];
    dec.quat[4 * g] = q[0]; dec.quat[4 * g + 1] = q[1]; dec.quat[4 * g + 2] = q[2]; dec.quat[4 * g + 3] = q[3];
  }
  if (rec) project_gaussian(b, v, mu, s, q, op, col, rec + g * kRecF4, counts + g, keys + g, err, mu_lo);
}

}  // namespace pgs
