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
// Two kernels.  k_decode_mlp_tc: one CTA of 384 threads decodes 128 visible
// (view, anchor) rows at a time.  Threads 0-127 own one row each for the
// operands and layer 1; after layer 2, warps w, w + 4, w + 8 share the 32 rows
// of TMEM lane quarter w and store layer-2 columns 0-31 (colour), 32-79 and
// 80-111, biases added, as Eq. 4's 110 outputs of the row into the row scratch
// (blocks of 32 rows, feature-major).  Operands use the no-swizzle K-major
// core-matrix layout; one elected thread issues the MMAs.  Every wait on the
// MMA barrier is bounded; on a timeout the kernel raises PGS_ERR_TIMEOUT, waits
// once more, frees its tensor memory and returns.
// k_project_decoded: the activations and the EWA projection of every decoded
// Gaussian, one thread per Gaussian, a 32-row block of outputs staged in shared
// memory per CTA.  Split from the MMA kernel, the projection (about 2,000
// instructions per Gaussian) runs at the occupancy its registers allow instead
// of behind the MMA kernel's shared-memory and tensor-memory footprint.
#include "pgs_decode_tc.cuh"

namespace pgs {

using namespace tc;

constexpr int kTcThreads = 384;
constexpr uint32_t kTmemCols = 256;         // D1 at column 0, D2 at column 32
size_t decode_tc_smem_bytes() { return sizeof(DecSmem) + 1024; }

// layer-2 columns [c0, c0 + 16 n) of this thread's row, biases added, into the row scratch
template <int N16>
__device__ __forceinline__ void store_l2_columns(uint32_t tlane, int c0, const float* b2p, bool valid, long long r,
                                                 float* __restrict__ zout) {
#pragma unroll
  for (int u = 0; u < N16; ++u) {
    float v[16];
    tmem_ld16(tlane + kD2Col + c0 + 16 * u, v);
    if (!valid) continue;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int n = c0 + 16 * u + i, o = l2_out(n);
      if (o >= 0) zout[sc_at(r, o, kOut)] = v[i] + b2p[n];
    }
  }
}

template <bool kSplit>
__global__ void __launch_bounds__(kTcThreads, 2) k_decode_mlp_tc(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A,
                                                       pgs_mlp_ptrs Wt, const uint32_t* __restrict__ rows,
                                                       const long long* __restrict__ n_rows_p, long long cap,
                                                       float* __restrict__ zout, uint32_t* err) {
  extern __shared__ unsigned char smem_raw[];
  DecSmem& sm = *reinterpret_cast<DecSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool row_thread = tid < kRows;                // operand rows and layer 1
  const int erow = (warp & 3) * 32 + (tid & 31);      // the row whose outputs this thread stores
  const int epart = warp >> 2;                        // 0: columns 0-31, 1: 32-79, 2: 80-111
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
    const long long r = tile * kRows + erow;
    const bool valid = r < n_rows;
    if (epart == 0) store_l2_columns<2>(tlane, 0, sm.b2p, valid, r, zout);
    else if (epart == 1) store_l2_columns<3>(tlane, 32, sm.b2p, valid, r, zout);
    else store_l2_columns<2>(tlane, 80, sm.b2p, valid, r, zout);
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

// One CTA per 32-row block of the row scratch at a time: the block's 110 x 32
// outputs are staged in shared memory (rows padded to 33 words: the ten
// Gaussians of a row read different banks), then thread t takes Gaussian
// j = t % 10 of row t / 10, so a warp's records, counts and keys are consecutive.
constexpr int kProjThreads = 10 * kScBlock;
__global__ void __launch_bounds__(kProjThreads, 3) k_project_decoded(const __grid_constant__ BatchDev b,
                                                                   pgs_anchor_ptrs A,
                                                                   const uint32_t* __restrict__ rows,
                                                                   const long long* __restrict__ n_rows_p,
                                                                   long long cap, const float* __restrict__ zin,
                                                                   float4* __restrict__ rec,
                                                                   uint32_t* __restrict__ counts,
                                                                   uint32_t* __restrict__ keys, DecodeOut dec,
                                                                   uint32_t* err) {
  __shared__ float s_z[kOut * (kScBlock + 1)];
  const long long n_rows = min(*n_rows_p, cap);
  const long long n_blk = (n_rows + kScBlock - 1) / kScBlock;
  const int lr = threadIdx.x / kNOff, j = threadIdx.x % kNOff;
  for (long long blk = blockIdx.x; blk < n_blk; blk += gridDim.x) {
    __syncthreads();
    const float* src = zin + (size_t)blk * kOut * kScBlock;
    for (int i = threadIdx.x; i < kOut * kScBlock; i += kProjThreads)
      s_z[(i / kScBlock) * (kScBlock + 1) + i % kScBlock] = src[i];
    __syncthreads();
    const long long r = blk * kScBlock + lr;
    if (r >= n_rows) continue;
    const uint32_t rw = rows[r];
    const int vi = rw >> 27;
    const long long a = rw & ((1u << 27) - 1);
    const float l[3] = {expf(A.log_l[3 * a]), expf(A.log_l[3 * a + 1]), expf(A.log_l[3 * a + 2])};
    const float xa[3] = {A.x[3 * a], A.x[3 * a + 1], A.x[3 * a + 2]};
    // Eq. 4's blocked outputs of Gaussian j: opacity j, colour 10 + 3j, scale 40 + 3j, quaternion 70 + 4j
    const int of[11] = {j, 10 + 3 * j, 11 + 3 * j, 12 + 3 * j, 40 + 3 * j, 41 + 3 * j, 42 + 3 * j,
                        70 + 4 * j, 71 + 4 * j, 72 + 4 * j, 73 + 4 * j};
    float z[11];
#pragma unroll
    for (int t = 0; t < 11; ++t) z[t] = s_z[of[t] * (kScBlock + 1) + lr];
    decode_gaussian(b, b.v[vi], z, l, xa, A.offsets + (a * kNOff + j) * 3, r * kNOff + j, rec, counts, keys, dec,
                    err);
  }
}

cudaError_t launch_decode_project_tc(bool split, const BatchDev& b, const pgs_anchor_ptrs& A, const pgs_mlp_ptrs& W,
                                     const uint32_t* rows, const long long* n_rows, long long cap, float* zbuf,
                                     float4* rec, uint32_t* counts, uint32_t* keys, const DecodeOut& dec,
                                     uint32_t* err, cudaStream_t st) {
  const size_t smem = decode_tc_smem_bytes();
  const void* k = split ? reinterpret_cast<const void*>(k_decode_mlp_tc<true>)
                        : reinterpret_cast<const void*>(k_decode_mlp_tc<false>);
  const int per_sm = prepare_smem_kernel(k, kTcThreads, smem);
  const int sms = device_sm_count();
  const long long tiles = (cap + kRows - 1) / kRows;
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)per_sm * sms));
  if (split)
    k_decode_mlp_tc<true><<<grid, kTcThreads, smem, st>>>(b, A, W, rows, n_rows, cap, zbuf, err);
  else
    k_decode_mlp_tc<false><<<grid, kTcThreads, smem, st>>>(b, A, W, rows, n_rows, cap, zbuf, err);
  const int per_sm_p = resident_ctas_per_sm(reinterpret_cast<const void*>(k_project_decoded), kProjThreads);
  const long long blocks = (cap + kScBlock - 1) / kScBlock;
  const int grid_p = (int)std::max<long long>(1, std::min<long long>(blocks, (long long)per_sm_p * sms));
  k_project_decoded<<<grid_p, kProjThreads, 0, st>>>(b, A, rows, n_rows, cap, zbuf, rec, counts, keys, dec, err);
  return cudaGetLastError();
}

}  // namespace pgs
