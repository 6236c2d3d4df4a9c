// Projective TSDF fusion of rendered depth and colour (the supplementary's mesh
// reconstruction: voxel 0.01 and truncation 0.04 for the aerial scenes).
//
// One thread per voxel, threads walking the volume in 8 x 8 x 8 bricks with the
// bricks of a column (z) consecutive: the voxels in flight at any time form a
// few compact columns, so their projections touch a small part of each view and
// the pixel reads hit in L2 more often (a slab order sweeps whole images per
// layer; at 0.01 voxels about 7 px apart, neighbouring voxels share no sector).
// On the aerial batch this cut the DRAM reads from 7.8 to 2.4 GB per launch;
// groups of 4 x 4 x 4 bricks read 2.2 GB but ran no faster.  A warp covers 4
// rows of 8 consecutive x of one brick.  The voxel's running state is
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

constexpr int kTsdfGroup = 4;   // views projected (and their pixels fetched) together
constexpr int kBrick = 8;       // voxels per brick edge (a brick is 512 consecutive threads)
static_assert(kBrick * kBrick * kBrick == 512, "the thread index splits as brick << 9 | voxel in brick");

// Depth and colour of every pixel interleaved as one 16-byte record (D, r, g, b): a
// voxel-view sample then reads one 32-byte sector instead of four (the depth plane
// and three colour planes), since voxels sit several pixels apart in the views.
__global__ void __launch_bounds__(256) k_tsdf_pack(const __grid_constant__ BatchDev b, const float* __restrict__ depth,
                                                   const float* __restrict__ rgb, float4* __restrict__ packed) {
  int vi = 0;   // threads walk increasing pixel indices, so the view only moves forward
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < b.total_pixels;
       p += (long long)gridDim.x * blockDim.x) {
    while (vi + 1 < b.n_views && p >= b.v[vi + 1].pix_off) ++vi;
    const ViewDev& w = b.v[vi];
    const long long HW = (long long)w.W * w.H;
    const long long p3 = 2 * w.pix_off + p;
    packed[p] = make_float4(__ldg(depth + p), __ldg(rgb + p3), __ldg(rgb + p3 + HW), __ldg(rgb + p3 + 2 * HW));
  }
}

// packed: the maps interleaved by k_tsdf_pack (with colour), or null to read the planes
__global__ void __launch_bounds__(256) k_tsdf_integrate(const __grid_constant__ BatchDev b, TsdfArgs a,
                                                        const float* __restrict__ depth,
                                                        const float* __restrict__ rgb,
                                                        const float4* __restrict__ packed, float* __restrict__ tsdf,
                                                        float* __restrict__ weight, float* __restrict__ color) {
  const long long nxy = (long long)a.dims[0] * a.dims[1];
  const int nbx = (a.dims[0] + kBrick - 1) / kBrick, nby = (a.dims[1] + kBrick - 1) / kBrick;
  const int nbz = (a.dims[2] + kBrick - 1) / kBrick;
  const long long n_threads = (long long)nbx * nby * nbz * (kBrick * kBrick * kBrick);
  const float itrunc = 1.f / a.trunc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_threads;
       t += (long long)gridDim.x * blockDim.x) {
    const unsigned brick = (unsigned)(t >> 9);   // fewer than 2^25 bricks (checked by the host)
    const int w = (int)(t & 511);
    const int bz = (int)(brick % (unsigned)nbz);
    const unsigned rest = brick / (unsigned)nbz;
    const int bx = (int)(rest % (unsigned)nbx), by = (int)(rest / (unsigned)nbx);
    const int i = bx * kBrick + (w & 7), j = by * kBrick + ((w >> 3) & 7), k = bz * kBrick + (w >> 6);
    if (i >= a.dims[0] || j >= a.dims[1] || k >= a.dims[2]) continue;
    const long long idx = (long long)k * nxy + (long long)j * a.dims[0] + i;
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
    for (int v0 = 0; v0 < b.n_views; v0 += kTsdfGroup) {
      // project the centre into a group of views and fetch their pixels before any update,
      // so the gathers of the group are in flight together
      float zc[kTsdfGroup], dd[kTsdfGroup], cc[kTsdfGroup][3];
#pragma unroll
      for (int t = 0; t < kTsdfGroup; ++t) {
        zc[t] = 0.f;
        dd[t] = 0.f;
        cc[t][0] = cc[t][1] = cc[t][2] = 0.f;
        const int v = v0 + t;
        if (v >= b.n_views) continue;
        const ViewDev& w = b.v[v];
        const float z = fmaf(w.R[6], X[0], fmaf(w.R[7], X[1], fmaf(w.R[8], X[2], w.t[2])));
        if (!(z > b.p.near_plane)) continue;
        const float x = fmaf(w.R[0], X[0], fmaf(w.R[1], X[1], fmaf(w.R[2], X[2], w.t[0])));
        const float y = fmaf(w.R[3], X[0], fmaf(w.R[4], X[1], fmaf(w.R[5], X[2], w.t[1])));
        const float iz = rcp_approx(z);
        const float fu = floorf(fmaf(w.fx * x, iz, w.cx)), fv = floorf(fmaf(w.fy * y, iz, w.cy));
        if (!(fu >= 0.f && fv >= 0.f && fu <= (float)(w.W - 1) && fv <= (float)(w.H - 1))) continue;
        const long long p = w.pix_off + (long long)((int)fv * w.W + (int)fu);
        zc[t] = z;
        if (packed) {
          const float4 q = __ldg(packed + p);
          dd[t] = q.x;
          cc[t][0] = q.y;
          cc[t][1] = q.z;
          cc[t][2] = q.w;
        } else {
          dd[t] = __ldg(depth + p);
          if (color) {
            const long long HW = (long long)w.W * w.H;
            const long long p3 = 2 * w.pix_off + p;
            cc[t][0] = __ldg(rgb + p3);
            cc[t][1] = __ldg(rgb + p3 + HW);
            cc[t][2] = __ldg(rgb + p3 + 2 * HW);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < kTsdfGroup; ++t) {
        const float sdf = dd[t] - zc[t];
        if (!(dd[t] > 0.f) || sdf < -a.trunc) continue;    // no pixel, no depth, or behind the band
        const float obs = fminf(1.f, sdf * itrunc);
        const float W1 = W + 1.f, iw = rcp_approx(W1);
        T = fmaf(T, W, obs) * iw;
        if (color) {
          C0 = fmaf(C0, W, cc[t][0]) * iw;
          C1 = fmaf(C1, W, cc[t][1]) * iw;
          C2 = fmaf(C2, W, cc[t][2]) * iw;
        }
        W = W1;
        changed = true;
      }
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

int launch_tsdf(const BatchDev& b, const TsdfArgs& a, const float* depth, const float* rgb, float4* pack_scratch,
                float* tsdf, float* weight, float* color, int num_sms, cudaStream_t st) {
  const long long nb = (long long)((a.dims[0] + 7) / 8) * ((a.dims[1] + 7) / 8) * ((a.dims[2] + 7) / 8);
  if (nb <= 0) return 0;
  int launches = 0;
  const float4* packed = nullptr;
  if (rgb && pack_scratch) {
    k_tsdf_pack<<<num_sms * 8, 256, 0, st>>>(b, depth, rgb, pack_scratch);
    packed = pack_scratch;
    ++launches;
  }
  const long long blk = std::min<long long>(nb * 2, (long long)num_sms * 16);
  k_tsdf_integrate<<<(unsigned)blk, 256, 0, st>>>(b, a, depth, rgb, packed, tsdf, weight, color);
  return launches + 1;
}

}  // namespace pgs
