// Shared decoder F_de (Eq. 4) on the 5th-generation tensor cores: BF16
// operands, FP32 accumulation in tensor memory, the activation / projection
// epilogue fused behind it.
//
// Precision per output head, chosen from how each head's error reaches the
// images.  A colour enters the image through a sigmoid (gain <= 1/4) and one
// BF16 pass moves it by < 1e-3.  The opacity, scale and rotation heads decide
// the normal of Eq. 6 and the depth of Eq. 7 through the blending weights, the
// smallest-scale axis (an argmin) and the normalisation of a 4-vector that can
// be short; one BF16 pass moves those maps by up to ~7e-2.  So:
//   layer 1  D1[128 x 32]  = X . W1^T            three-piece BF16 split of X
//                                                 and W1, six products (FP32-accurate)
//   layer 2  colour block   D2[:, 0..31]  = bf16(H) . bf16(W2_colour)^T   one pass
//            shape block    D2[:, 32..111] = H . W2_shape^T                 six products
// where a three-piece split x = p0 + p1 + p2 (BF16 each) is exact for FP32 x
// and the products p_i q_j with i + j <= 2 leave out terms below 2^-24 |xq|.
// The one-pass form (every product p0 q0, as a study of BF16 error) is the
// kSplit = false instantiation.
//
// One CTA of 384 threads decodes 128 visible (view, anchor) rows at a time.
// Threads 0-127 own one row each for the operands and layer 1; after layer 2,
// warps w, w + 4, w + 8 share the 32 rows of TMEM lane quarter w and take
// Gaussians 0-3, 4-7 and 8-9 of each row.  Operands use the no-swizzle K-major
// core-matrix layout; one elected thread issues the MMAs.  Every wait on the
// MMA barrier is bounded; on a timeout the kernel raises PGS_ERR_TIMEOUT, waits
// once more, frees its tensor memory and returns.
#include "pgs_decode_tc.cuh"

namespace pgs {

using namespace tc;

constexpr int kTcThreads = 384;
constexpr uint32_t kTmemCols = 256;         // D1 at column 0, D2 at column 32
size_t decode_tc_smem_bytes() { return sizeof(DecSmem) + 1024; }

// epilogue of part P (Gaussians 4P .. 4P + 3, or 8 .. 9) of this thread's row
template <int P>
__device__ __forceinline__ void decode_tc_epilogue(const BatchDev& b, const pgs_anchor_ptrs& A, uint32_t tlane,
                                                   const float* b2p, bool valid, int vi, long long a, long long r,
                                                   const float (&l)[3], const float (&xa)[3], float4* rec,
                                                   uint32_t* counts, uint32_t* keys, const DecodeOut& dec,
                                                   uint32_t* err) {
  constexpr int nG = P == 2 ? 2 : 4;
  float cz[3 * nG];
  dec_load_colour<P, nG>(tlane, cz);
  // shape blocks, two Gaussians (16 columns) per load
#pragma unroll
  for (int u2 = 0; u2 < nG / 2; ++u2) {
    float sz[16];
    tmem_ld16(tlane + kD2Col + kShape0 + 32 * P + 16 * u2, sz);
    if (!valid) continue;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int u = 2 * u2 + w, j = 4 * P + u;
      float z[11];
      dec_outputs(b2p, j, cz + 3 * u, sz + 8 * w, z);
      decode_gaussian(b, b.v[vi], z, l, xa, A.offsets + (a * kNOff + j) * 3, r * kNOff + j, rec, counts, keys, dec,
                      err);
    }
  }
}

template <bool kSplit>
__global__ void __launch_bounds__(kTcThreads, 2) k_decode_project_tc(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A,
                                                           pgs_mlp_ptrs Wt, const uint32_t* __restrict__ rows,
                                                           const long long* __restrict__ n_rows_p, long long cap,
                                                           float4* __restrict__ rec, uint32_t* __restrict__ counts,
                                                           uint32_t* __restrict__ keys, DecodeOut dec, uint32_t* err) {
  extern __shared__ unsigned char smem_raw[];
  DecSmem& sm = *reinterpret_cast<DecSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool row_thread = tid < kRows;                // operand rows and layer 1
  const int erow = (warp & 3) * 32 + (tid & 31);      // the row whose Gaussians this thread projects
  const int epart = warp >> 2;                        // 0: Gaussians 0-3, 1: 4-7, 2: 8-9
  constexpr int kPieces = kSplit ? 3 : 1;
  dec_stage_weights(sm, Wt, b.p.in_dim, kPieces);
  const uint32_t mbar = smem_u32(&sm.mbar);
  if (tid == 0) mbar_init(mbar);
  if (warp == 0) tmem_alloc(&sm.tmem_base, kTmemCols);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.tmem_base;
  const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  const long long n_rows = min(*n_rows_p, cap);
  const long long n_tiles = (n_rows + kRows - 1) / kRows;
  uint32_t phase = 0;
  bool timed_out = false;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    if (row_thread) {
      float X[kMaxIn];
      dec_stage_x(sm, b, A, rows, tile * kRows + tid, n_rows, tid, kPieces, X);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      dec_issue_layer1(sm, tmem, kSplit);
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase))) { timed_out = true; break; }
    phase ^= 1u;
    fence_after();
    if (row_thread) {
      float h[kHidden];
      dec_stage_h(sm, tlane, tid, kPieces, h);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      dec_issue_layer2(sm, tmem, kSplit);
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase))) { timed_out = true; break; }
    phase ^= 1u;
    fence_after();
    // epilogue: this thread's row, Gaussians of its part
    const long long r = tile * kRows + erow;
    const bool valid = r < n_rows;
    int vi = 0;
    long long a = 0;
    float l[3] = {1.f, 1.f, 1.f}, xa[3] = {0.f, 0.f, 0.f};
    if (valid) {
      const uint32_t rw = rows[r];
      vi = rw >> 27;
      a = rw & ((1u << 27) - 1);
      l[0] = expf(A.log_l[3 * a]); l[1] = expf(A.log_l[3 * a + 1]); l[2] = expf(A.log_l[3 * a + 2]);
      xa[0] = A.x[3 * a]; xa[1] = A.x[3 * a + 1]; xa[2] = A.x[3 * a + 2];
    }
    if (epart == 0) decode_tc_epilogue<0>(b, A, tlane, sm.b2p, valid, vi, a, r, l, xa, rec, counts, keys, dec, err);
    else if (epart == 1) decode_tc_epilogue<1>(b, A, tlane, sm.b2p, valid, vi, a, r, l, xa, rec, counts, keys, dec, err);
    else decode_tc_epilogue<2>(b, A, tlane, sm.b2p, valid, vi, a, r, l, xa, rec, counts, keys, dec, err);
    fence_before();
    __syncthreads();
  }
  if (timed_out) {
    if (tid == 0) set_flag(err, kFlagTimeout);
    (void)mbar_wait(mbar, phase);   // let the MMA in flight finish before the memory is released
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

cudaError_t launch_decode_project_tc(bool split, const BatchDev& b, const pgs_anchor_ptrs& A, const pgs_mlp_ptrs& W,
                                     const uint32_t* rows, const long long* n_rows, long long cap, float4* rec,
                                     uint32_t* counts, uint32_t* keys, const DecodeOut& dec, uint32_t* err,
                                     cudaStream_t st) {
  const size_t smem = decode_tc_smem_bytes();
  const void* k = split ? reinterpret_cast<const void*>(k_decode_project_tc<true>)
                        : reinterpret_cast<const void*>(k_decode_project_tc<false>);
  const int per_sm = prepare_smem_kernel(k, kTcThreads, smem);
  const long long tiles = (cap + kRows - 1) / kRows;
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)per_sm * device_sm_count()));
  if (split)
    k_decode_project_tc<true><<<grid, kTcThreads, smem, st>>>(b, A, W, rows, n_rows, cap, rec, counts, keys, dec, err);
  else
    k_decode_project_tc<false><<<grid, kTcThreads, smem, st>>>(b, A, W, rows, n_rows, cap, rec, counts, keys, dec, err);
  return cudaGetLastError();
}

}  // namespace pgs
