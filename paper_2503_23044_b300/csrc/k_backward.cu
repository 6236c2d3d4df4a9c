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
#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }

struct ProjGrad {
  float dmu[3], ds[3], dq[4], dop, dcol[3];
};

// Chain the 13 per-Gaussian-view gradients back to (mu, s, unit q, opacity, colour).
__device__ void project_backward(const BatchDev& b, const ViewDev& v, const float mu[3], const float s[3],
                                 const float q[4], const float* gr, ProjGrad& out) {
  const ParamsDev& p = b.p;
  const float* W = v.R;
  const float x = W[0] * mu[0] + W[1] * mu[1] + W[2] * mu[2] + v.t[0];
  const float y = W[3] * mu[0] + W[4] * mu[1] + W[5] * mu[2] + v.t[1];
  const float z = W[6] * mu[0] + W[7] * mu[1] + W[8] * mu[2] + v.t[2];
  const float iz = 1.f / z, iz2 = iz * iz;
  const float xz = x * iz, yz = y * iz;
  const bool clx = xz < -v.lim_x || xz > v.lim_x, cly = yz < -v.lim_y || yz > v.lim_y;
  const float txz = fminf(fmaxf(xz, -v.lim_x), v.lim_x), tyz = fminf(fmaxf(yz, -v.lim_y), v.lim_y);
  const float J00 = v.fx * iz, J02 = -v.fx * txz * iz, J11 = v.fy * iz, J12 = -v.fy * tyz * iz;
  float Rg[9];
  quat_to_rot(q[0], q[1], q[2], q[3], Rg);
  float T[2][3];
  for (int c = 0; c < 3; ++c) {
    T[0][c] = J00 * W[c] + J02 * W[6 + c];
    T[1][c] = J11 * W[3 + c] + J12 * W[6 + c];
  }
  float M[3][3];  // M = Rg diag(s)
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) M[i][k] = Rg[3 * i + k] * s[k];
  float U[2][3];  // U = T M
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < 3; ++k) U[r][k] = T[r][0] * M[0][k] + T[r][1] * M[1][k] + T[r][2] * M[2][k];
  float a = p.dilation, bb = 0.f, c = p.dilation;
  for (int k = 0; k < 3; ++k) {
    a += U[0][k] * U[0][k];
    bb += U[0][k] * U[1][k];
    c += U[1][k] * U[1][k];
  }
  const float det = a * c - bb * bb, idet = 1.f / det;
  const float QA = c * idet, QB = -bb * idet, QC = a * idet;
  // dL/dcov = -Q G Q, G = [[dA, dB/2],[dB/2, dC]]
  const float gA = gr[2], gB = 0.5f * gr[3], gC = gr[4];
  const float t00 = QA * gA + QB * gB, t01 = QA * gB + QB * gC;
  const float t10 = QB * gA + QC * gB, t11 = QB * gB + QC * gC;
  const float D00 = -(t00 * QA + t01 * QB), D01 = -(t00 * QB + t01 * QC), D11 = -(t10 * QB + t11 * QC);
  // dL/dU = 2 D U (D symmetric with off-diagonal D01)
  float dU[2][3];
  for (int k = 0; k < 3; ++k) {
    dU[0][k] = 2.f * (D00 * U[0][k] + D01 * U[1][k]);
    dU[1][k] = 2.f * (D01 * U[0][k] + D11 * U[1][k]);
  }
  // U = T M: dT = dU M^T, dM = T^T dU
  float dT[2][3], dM[3][3];
  for (int r = 0; r < 2; ++r)
    for (int cc = 0; cc < 3; ++cc) dT[r][cc] = dU[r][0] * M[cc][0] + dU[r][1] * M[cc][1] + dU[r][2] * M[cc][2];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) dM[i][k] = T[0][i] * dU[0][k] + T[1][i] * dU[1][k];
  // M = Rg diag(s)
  float dRg[9];
  for (int k = 0; k < 3; ++k) {
    out.ds[k] = dM[0][k] * Rg[k] + dM[1][k] * Rg[3 + k] + dM[2][k] * Rg[6 + k];
    for (int i = 0; i < 3; ++i) dRg[3 * i + k] = dM[i][k] * s[k];
  }
  // T = J W: dJ = dT W^T (entries (0,0), (0,2), (1,1), (1,2) are live)
  const float dJ00 = dT[0][0] * W[0] + dT[0][1] * W[1] + dT[0][2] * W[2];
  const float dJ02 = dT[0][0] * W[6] + dT[0][1] * W[7] + dT[0][2] * W[8];
  const float dJ11 = dT[1][0] * W[3] + dT[1][1] * W[4] + dT[1][2] * W[5];
  const float dJ12 = dT[1][0] * W[6] + dT[1][1] * W[7] + dT[1][2] * W[8];
  // camera-frame mean: 2D mean, J
  float dx = v.fx * iz * gr[0];
  float dy = v.fy * iz * gr[1];
  float dz = -v.fx * x * iz2 * gr[0] - v.fy * y * iz2 * gr[1];
  dz += -v.fx * iz2 * dJ00 - v.fy * iz2 * dJ11;
  if (clx) dz += v.fx * txz * iz2 * dJ02;
  else { dx += -v.fx * iz2 * dJ02; dz += 2.f * v.fx * x * iz2 * iz * dJ02; }
  if (cly) dz += v.fy * tyz * iz2 * dJ12;
  else { dy += -v.fy * iz2 * dJ12; dz += 2.f * v.fy * y * iz2 * iz * dJ12; }
  // normal n_c = sgn W Rg[:,k] and d = n_c . mu_c
  int k = 0;
  if (s[1] < s[k]) k = 1;
  if (s[2] < s[k]) k = 2;
  const float nw0 = Rg[k], nw1 = Rg[3 + k], nw2 = Rg[6 + k];
  float n0 = W[0] * nw0 + W[1] * nw1 + W[2] * nw2;
  float n1 = W[3] * nw0 + W[4] * nw1 + W[5] * nw2;
  float n2 = W[6] * nw0 + W[7] * nw1 + W[8] * nw2;
  const float sg = (n0 * x + n1 * y + n2 * z > 0.f) ? -1.f : 1.f;
  n0 *= sg; n1 *= sg; n2 *= sg;
  const float gd = gr[9];
  const float gn0 = gr[10] + gd * x, gn1 = gr[11] + gd * y, gn2 = gr[12] + gd * z;
  dx += gd * n0; dy += gd * n1; dz += gd * n2;
  // dRg[:,k] += sg W^T gn
  dRg[k] += sg * (W[0] * gn0 + W[3] * gn1 + W[6] * gn2);
  dRg[3 + k] += sg * (W[1] * gn0 + W[4] * gn1 + W[7] * gn2);
  dRg[6 + k] += sg * (W[2] * gn0 + W[5] * gn1 + W[8] * gn2);
  // world mean
  out.dmu[0] = W[0] * dx + W[3] * dy + W[6] * dz;
  out.dmu[1] = W[1] * dx + W[4] * dy + W[7] * dz;
  out.dmu[2] = W[2] * dx + W[5] * dy + W[8] * dz;
  // rotation matrix of a unit quaternion (w, x, y, z)
  const float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
  out.dq[0] = 2.f * (-qz * dRg[1] + qy * dRg[2] + qz * dRg[3] - qx * dRg[5] - qy * dRg[6] + qx * dRg[7]);
  out.dq[1] = 2.f * (qy * dRg[1] + qz * dRg[2] + qy * dRg[3] - 2.f * qx * dRg[4] - qw * dRg[5] + qz * dRg[6] +
                     qw * dRg[7] - 2.f * qx * dRg[8]);
  out.dq[2] = 2.f * (-2.f * qy * dRg[0] + qx * dRg[1] + qw * dRg[2] + qx * dRg[3] + qz * dRg[5] - qw * dRg[6] +
                     qz * dRg[7] - 2.f * qy * dRg[8]);
  out.dq[3] = 2.f * (-2.f * qz * dRg[0] - qw * dRg[1] + qx * dRg[2] + qw * dRg[3] - 2.f * qz * dRg[4] +
                     qy * dRg[5] + qx * dRg[6] + qy * dRg[7]);
  out.dop = gr[5];
  out.dcol[0] = gr[6]; out.dcol[1] = gr[7]; out.dcol[2] = gr[8];
}

// d normalise(q) -> d q_raw ; q_unit = q / |q| (identity substitute has no gradient)
__device__ __forceinline__ void quat_norm_backward(const float qr[4], float qn, const float dqu[4], float dq[4]) {
  if (qn < 1e-12f) { dq[0] = dq[1] = dq[2] = dq[3] = 0.f; return; }
  const float iq = 1.f / qn;
  const float u[4] = {qr[0] * iq, qr[1] * iq, qr[2] * iq, qr[3] * iq};
  const float dt = u[0] * dqu[0] + u[1] * dqu[1] + u[2] * dqu[2] + u[3] * dqu[3];
  for (int i = 0; i < 4; ++i) dq[i] = (dqu[i] - u[i] * dt) * iq;
}

__device__ __forceinline__ bool load_grad(const float* __restrict__ grad, long long g, float gr[13]) {
  const float4* p = reinterpret_cast<const float4*>(grad + g * 16);
  const float4 a = p[0], b = p[1], c = p[2], d = p[3];
  gr[0] = a.x; gr[1] = a.y; gr[2] = a.z; gr[3] = a.w;
  gr[4] = b.x; gr[5] = b.y; gr[6] = b.z; gr[7] = b.w;
  gr[8] = c.x; gr[9] = c.y; gr[10] = c.z; gr[11] = c.w;
  gr[12] = d.x;
  bool nz = false;
  for (int i = 0; i < 13; ++i) nz |= gr[i] != 0.f;
  return nz;
}

__device__ __forceinline__ void add_if(float* p, float v) {
  if (p && v != 0.f) atomicAdd(p, v);
}

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

// z = b2[o] + W2[o] . H (one decoder output, weight row read as float4)
__device__ __forceinline__ float w2_dot(const MlpSmemB& m, int o, const float (&H)[kHidden]) {
  const float4* w = reinterpret_cast<const float4*>(m.W2[o]);
  float acc = m.b2[o];
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
// Gaussian by Gaussian, dX = W1^T (dH . [H > 0]).
__global__ void __launch_bounds__(128) k_decode_bwd(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A,
                                                    pgs_mlp_ptrs Wt, const uint32_t* __restrict__ rows,
                                                    const long long* __restrict__ n_rows_p, long long cap,
                                                    const float* __restrict__ grad, pgs_param_grad_ptrs out,
                                                    float* __restrict__ sc_dZ, float* __restrict__ sc_H,
                                                    float* __restrict__ sc_dH, float* __restrict__ sc_X, uint32_t* err) {
  __shared__ MlpSmemB m;
  const int in_dim = b.p.in_dim;
  for (int t = threadIdx.x; t < kHidden * kMaxIn; t += blockDim.x) {
    const int i = t / kMaxIn, j = t % kMaxIn;
    m.W1[i][j] = j < in_dim ? Wt.W1[i * in_dim + j] : 0.f;
  }
  for (int t = threadIdx.x; t < kHidden; t += blockDim.x) m.b1[t] = Wt.b1[t];
  for (int t = threadIdx.x; t < kOut * kHidden; t += blockDim.x) m.W2[t / kHidden][t % kHidden] = Wt.W2[t];
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
        H[i] = fmaxf(acc, 0.f);
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
      for (int t = 0; t < 11; ++t) z[t] = w2_dot(m, idx[t], H);
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
                                                           int in_dim, float* __restrict__ partials) {
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
        for (int c = 0; c < 4; ++c) w[c] = sH[rr][gb + c];
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

void launch_mlp_wgrad(const float* dZ, const float* H, const float* dH, const float* X, const long long* n_rows,
                      long long cap, int in_dim, float* partials, int nb, const pgs_param_grad_ptrs& out,
                      cudaStream_t st) {
  k_mlp_wgrad_partial<<<nb, 256, 0, st>>>(dZ, H, dH, X, n_rows, cap, in_dim, partials);
  k_mlp_wgrad_final<<<(wgrad_outputs(in_dim) + 31) / 32, 256, 0, st>>>(partials, nb, in_dim, out);
}

}  // namespace pgs
