// Projective TSDF fusion of rendered depth and colour (the supplementary's mesh
// reconstruction: voxel 0.01 and truncation 0.04 for the aerial scenes).
//
// One thread per voxel, x fastest (so a warp reads 32 consecutive voxels of the
// volume and projects into neighbouring pixels).  The voxel's running state is
// read once, every view of the batch is fused in batch order, and the state is
// written once: per view, the voxel centre is projected (camera depth z > near
// plane), the nearest pixel (floor of the projection, pixel centres at +1/2)
// must lie in the frame with a rendered depth D > 0, sdf = D - z must be at
// least -trunc, and then T <- (T W + min(1, sdf / trunc)) / (W + 1), the colour
// likewise, W <- W + 1.
#include <algorithm>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

__global__ void __launch_bounds__(256) k_tsdf_integrate(const __grid_constant__ BatchDev b, TsdfArgs a,
                                                        const float* __restrict__ depth,
                                                        const float* __restrict__ rgb, float* __restrict__ tsdf,
                                                        float* __restrict__ weight, float* __restrict__ color) {
  const long long nxy = (long long)a.dims[0] * a.dims[1];
  const long long n = nxy * a.dims[2];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long k = idx / nxy;
    const long long r = idx - k * nxy;
    const int j = (int)(r / a.dims[0]), i = (int)(r - (long long)j * a.dims[0]);
    const float X[3] = {fmaf((float)i + 0.5f, a.voxel, a.origin[0]), fmaf((float)j + 0.5f, a.voxel, a.origin[1]),
                        fmaf((float)k + 0.5f, a.voxel, a.origin[2])};
    float T = tsdf[idx], W = weight[idx];
    float C0 = 0.f, C1 = 0.f, C2 = 0.f;
    if (color) {
      C0 = color[3 * idx];
      C1 = color[3 * idx + 1];
      C2 = color[3 * idx + 2];
    }
    bool changed = false;
    for (int v = 0; v < b.n_views; ++v) {
      const ViewDev& w = b.v[v];
      const float z = fmaf(w.R[6], X[0], fmaf(w.R[7], X[1], fmaf(w.R[8], X[2], w.t[2])));
      if (!(z > b.p.near_plane)) continue;
      const float x = fmaf(w.R[0], X[0], fmaf(w.R[1], X[1], fmaf(w.R[2], X[2], w.t[0])));
      const float y = fmaf(w.R[3], X[0], fmaf(w.R[4], X[1], fmaf(w.R[5], X[2], w.t[1])));
      const float u = fmaf(w.fx, x / z, w.cx), vv = fmaf(w.fy, y / z, w.cy);
      const float fu = floorf(u), fv = floorf(vv);
      if (!(fu >= 0.f && fv >= 0.f && fu <= (float)(w.W - 1) && fv <= (float)(w.H - 1))) continue;
      const long long p = w.pix_off + (long long)((int)fv * w.W + (int)fu);
      const float d = __ldg(depth + p);
      if (!(d > 0.f)) continue;
      const float sdf = d - z;
      if (sdf < -a.trunc) continue;
      const float obs = fminf(1.f, sdf / a.trunc);
      const float W1 = W + 1.f;
      T = (T * W + obs) / W1;
      if (color) {
        const long long HW = (long long)w.W * w.H;
        const long long p3 = 2 * w.pix_off + p;
        C0 = (C0 * W + __ldg(rgb + p3)) / W1;
        C1 = (C1 * W + __ldg(rgb + p3 + HW)) / W1;
        C2 = (C2 * W + __ldg(rgb + p3 + 2 * HW)) / W1;
      }
      W = W1;
      changed = true;
    }
    if (changed) {
      tsdf[idx] = T;
      weight[idx] = W;
      if (color) {
        color[3 * idx] = C0;
        color[3 * idx + 1] = C1;
        color[3 * idx + 2] = C2;
      }
    }
  }
}

void launch_tsdf(const BatchDev& b, const TsdfArgs& a, const float* depth, const float* rgb, float* tsdf,
                 float* weight, float* color, int num_sms, cudaStream_t st) {
  const long long n = (long long)a.dims[0] * a.dims[1] * a.dims[2];
  if (n <= 0) return;
  const long long blk = std::min<long long>((n + 255) / 256, (long long)num_sms * 16);
  k_tsdf_integrate<<<(unsigned)blk, 256, 0, st>>>(b, a, depth, rgb, tsdf, weight, color);
}

}  // namespace pgs
