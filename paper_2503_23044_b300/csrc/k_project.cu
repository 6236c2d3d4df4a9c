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
#include "pgs_project.cuh"

namespace pgs {

// ---------------------------------------------------------------- explicit Gaussians
__global__ void __launch_bounds__(256) k_project_explicit(const __grid_constant__ BatchDev b,
                                                          pgs_explicit_ptrs P, long long N, float4* __restrict__ rec,
                                                          uint32_t* __restrict__ counts,
                                                          uint32_t* __restrict__ keys, uint32_t* err) {
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
    project_gaussian(b, b.v[v], mu, s, q, op, col, rec + g * kRecF4, counts + g, keys + g, err);
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

__global__ void __launch_bounds__(256) k_decode_project(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A,
                                                        pgs_mlp_ptrs Wt, const uint32_t* __restrict__ rows,
                                                        const long long* __restrict__ n_rows_p, long long cap,
                                                        float4* __restrict__ rec, uint32_t* __restrict__ counts,
                                                        uint32_t* __restrict__ keys, DecodeOut dec, uint32_t* err) {
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
      const long long g = r * kNOff + j;
      decode_gaussian(b, v, z, l, xa, A.offsets + (a * kNOff + j) * 3, g, rec, counts, keys, dec, err);
    }
  }
}

}  // namespace pgs
