// Per-Gaussian backward pieces shared by the decoder backward kernels: the
// projection backward (EWA projection, normal and plane distance of Eq. 6-7
// walked back to mean, scale, unit rotation, opacity and colour), the
// quaternion normalisation backward, the gradient-record load and a guarded
// atomic add.
#pragma once
#include "pgs_internal.cuh"

namespace pgs {

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }

struct ProjGrad {
  float dmu[3], ds[3], dq[4], dop, dcol[3];
};

// Chain the 13 per-Gaussian-view gradients back to (mu, s, unit q, opacity, colour).
__device__ inline void project_backward(const BatchDev& b, const ViewDev& v, const float mu[3], const float s[3],
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

}  // namespace pgs
