// Kernel entry points and launch helpers shared between the translation units.
#pragma once
#include "pgs_internal.cuh"

namespace pgs {

constexpr int kScanBlocks = 592;   // 4 x 148 SMs
constexpr int kLossBlocks = 1184;  // 8 x 148 SMs
// kernels enqueued by the multi-kernel launch helpers
constexpr int kScanLaunches = 3, kLossLaunches = 3, kWgradLaunches = 2;
constexpr int kPriorBlocks = 64, kPriorLaunches = 5, kPriorMaxK = 4;
constexpr int kNccLaunches = 4;
constexpr int kNccDone = kMaxViews / 2;   // index of the finished-blocks counter after the per-pair counts
constexpr int kNccChunks = 16;            // loss-reduction blocks per pair
constexpr float kNccInvalid = -2.f;   // NCC of a patch that is not used (NCC itself lies in [-1, 1])

// batch geometric NCC: weight of the loss, the variance guard and the stop-gradient form
struct NccArgs {
  float lambda, eps;
  int geometric;
};

// enhanced depth prior: the k nearest batch views of each view (-1 = none) and the filter threshold
struct PriorArgs {
  int nbr[kMaxViews][kPriorMaxK];
  int k;
  float tau_d;
};

struct DecodeOut {
  float *mu, *opacity, *color, *scale, *quat;
};

struct SortScratch {
  uint32_t* hist;
  uint32_t* counters;
  uint32_t* err;
  uint32_t* status;
  long long max_tiles;
  int radix_bits_max;   // 8, or 9 when the status arrays have room for 512 digits per tile
  size_t bytes;
};

// pgs_api.cu: message returned by pgs_last_error() on this host thread
void set_last_error(const char* msg);
// pgs_api.cu: resident CTAs per SM of `kernel` at `threads` threads (dynamic shared memory `smem`) on the
// current device, at least 1.  Queried once per (device, kernel, threads, smem) and cached; thread-safe.
// carveout >= 0 first sets the kernel's preferred shared-memory carveout (percent) on that device.
int resident_ctas_per_sm(const void* kernel, int threads, size_t smem = 0, int carveout = -1);
// pgs_api.cu: SM count of the current device (cached per device; thread-safe)
int device_sm_count();
// pgs_api.cu: allow `smem` bytes of dynamic shared memory for `kernel` on the current device (once per device)
// and return its resident CTAs per SM at `threads` threads
int prepare_smem_kernel(const void* kernel, int threads, size_t smem);

// k_project.cu
__global__ void k_project_explicit(const __grid_constant__ BatchDev b, pgs_explicit_ptrs P, long long N, float4* rec,
                                   uint32_t* counts, uint32_t* keys, uint32_t* err);
__global__ void k_anchor_cull(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A, long long Na, uint32_t* flags);
__global__ void k_compact_rows(const uint32_t* flags, const uint32_t* offs, long long total, long long Na,
                               uint32_t* rows, long long cap, uint32_t* err);
__global__ void k_decode_project(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A, pgs_mlp_ptrs Wt,
                                 const uint32_t* rows, const long long* n_rows_p, long long cap, float4* rec,
                                 uint32_t* counts, uint32_t* keys, DecodeOut dec, uint32_t* err);

// k_decode_tc.cu: the tensor-core decoder + projection; split = true is the production precision (layer 1 and
// the opacity / scale / rotation heads FP32-accurate, colour heads one BF16 pass), false the one-pass study form.
// zbuf: the decoded outputs pass through it (the row scratch layout, kOut features, at least sc_rows(cap) rows).
size_t decode_tc_smem_bytes();
cudaError_t launch_decode_project_tc(bool split, const BatchDev& b, const pgs_anchor_ptrs& A, const pgs_mlp_ptrs& W,
                                     const uint32_t* rows, const long long* n_rows, long long cap, float* zbuf,
                                     float4* rec, uint32_t* counts, uint32_t* keys, const DecodeOut& dec,
                                     uint32_t* err, cudaStream_t st);

// k_sort.cu
void launch_exclusive_scan(const uint32_t* in, const uint32_t* index, uint32_t* out, unsigned long long* total,
                           const long long* d_n, unsigned long long* sums, cudaStream_t st);
// keys per onesweep tile; the scratch layout below holds two look-back status
// arrays of (n_max / kSortTileKeys + 1) x (1 << radix_bits_max) words after the histograms
// (radix_bits_max 9 lets ranges of 17-18 bits sort in two 9-bit passes instead of three 8-bit ones)
constexpr int kSortTileKeys = 4096;
constexpr size_t sort_scratch_bytes_for(long long n_max, int radix_bits_max = 8) {
  return (size_t)(4 * 256 + 8) * 4 +
         (size_t)2 * ((n_max + kSortTileKeys - 1) / kSortTileKeys + 1) * (size_t)(1 << radix_bits_max) * 4;
}
SortScratch sort_scratch_layout(void* base, long long n_max, int radix_bits_max = 8);
int sort_passes(int bit_lo, int bit_hi);
// hold_tile: failure-path test hook (kNoHoldTile in production): that onesweep tile never publishes its
// look-back status, so the next tile's bounded wait runs out and raises kFlagTimeout.
constexpr uint32_t kNoHoldTile = 0xffffffffu;
cudaError_t launch_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                              const long long* d_n, long long n_max, int bit_lo, int bit_hi, const SortScratch& s,
                              uint32_t* err, uint32_t spin_limit, uint32_t hold_tile, int num_sms, cudaStream_t st,
                              int* n_launch = nullptr);
__global__ void k_sort_timeout_guard(const uint32_t* flags, long long* d_n, long long n_max, uint32_t* vals);
__global__ void k_emit_pairs(const __grid_constant__ BatchDev b, const float4* rec, const uint32_t* counts,
                             const uint32_t* sorted_g, const uint32_t* offs, const long long* d_ng, long long cap,
                             int mode, long long n_explicit, const uint32_t* rows, uint32_t* tiles_out,
                             uint32_t* g_out, uint32_t* err);
__global__ void k_pairs_total(const unsigned long long* total, long long cap, long long* d_p, uint32_t* err);
__global__ void k_tile_ranges(const uint32_t* tiles, const long long* d_p, uint2* ranges, int n_tiles, uint32_t* err);

// k_blend.cu (persistent kernels: tiles taken from a queue in `order` via `ctr`, which must start at 0)
bool launch_blend_fwd(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                      const pgs_image_ptrs& o, const uint32_t* order, uint32_t* ctr, cudaStream_t st);
bool launch_blend_bwd(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                      const pgs_image_ptrs& img, const pgs_image_grad_ptrs& gi, float* grad, const uint32_t* order,
                      uint32_t* ctr, cudaStream_t st);
__global__ void k_tile_order_keys(const uint2* ranges, int n_tiles, uint32_t* keys, uint32_t* vals);

// k_loss.cu
void launch_loss(const BatchDev& b, const pgs_image_ptrs& img, const pgs_target_ptrs& tgt, const pgs_loss_params& lp,
                 float* loss, const pgs_image_grad_ptrs& g, uint32_t* counts, float* partials, uint32_t* err,
                 cudaStream_t st);

// Decoder backward row scratch (dZ, H, dH, X per visible row): rows in blocks of
// kScBlock, feature-major inside a block, so a warp's 32 consecutive rows write
// one contiguous run per feature and a block of rows is one contiguous chunk.
constexpr int kScBlock = 32;
__host__ __device__ __forceinline__ size_t sc_at(long long r, int f, int width) {
  return ((size_t)(r / kScBlock) * width + f) * kScBlock + (size_t)(r % kScBlock);
}
__host__ __device__ __forceinline__ long long sc_rows(long long cap) { return (cap + kScBlock - 1) / kScBlock * kScBlock; }

// k_prior.cu
cudaError_t launch_ncc(const BatchDev& b, const NccArgs& a, const unsigned* centers, long long n_per, int n_pairs,
                       const float* rgb, const float* depth, const float* normal, float* ncc, float* loss,
                       float* g_rgb, float* g_depth, float* g_normal, void* scratch, float* luma, int num_sms,
                       cudaStream_t st);
size_t ncc_scratch_bytes();
// TSDF fusion: the volume and the truncation band
struct TsdfArgs {
  float origin[3], voxel, trunc;
  int dims[3];
};
// pack_scratch: 16 B per pixel of the batch for the interleaved maps, or null (colour fusion then reads the
// planes); returns the number of launches
int launch_tsdf(const BatchDev& b, const TsdfArgs& a, const float* depth, const float* rgb, float4* pack_scratch,
                float* tsdf, float* weight, float* color, int num_sms, cudaStream_t st);
void launch_prior_filter(const BatchDev& b, const PriorArgs& pa, const float* dp, const float* pts, long long n_pts,
                         float* partials, float* means, float* scale_shift, float* prior_out, float* mask_out,
                         float* err_out, int num_sms, cudaStream_t st);

// k_backward.cu
__global__ void k_project_bwd_explicit(const __grid_constant__ BatchDev b, pgs_explicit_ptrs P, long long N,
                                       const float* grad, pgs_param_grad_ptrs out, uint32_t* err);
__global__ void k_decode_bwd(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A, pgs_mlp_ptrs Wt,
                             const uint32_t* rows, const long long* n_rows_p, long long cap, const float* grad,
                             pgs_param_grad_ptrs out, float* sc_dZ, float* sc_H, float* sc_dH, float* sc_X,
                             uint32_t* err);
int mlp_wgrad_outputs(int in_dim);
// fixed-order sum of nb partial rows of the decoder weight gradients into out (accumulated)
cudaError_t launch_mlp_wgrad_final(const float* partials, int nb, int in_dim, const pgs_param_grad_ptrs& out,
                                   cudaStream_t st);
// k_decode_bwd_tc.cu: the decoder weight gradients of PGS_DECODE_BF16 on the tensor cores from the row scratch
// (at most nb_max partial rows)
cudaError_t launch_mlp_wgrad_tc(const float* dZ, const float* H, const float* dH, const float* X,
                                const long long* n_rows, long long cap, int in_dim, float* partials, int nb_max,
                                const pgs_param_grad_ptrs& out, uint32_t* err, cudaStream_t st);
// k_decode_bwd_tc.cu: the decoder backward of PGS_DECODE_BF16 on the tensor cores (fills the same row scratch)
cudaError_t launch_decode_bwd_tc(const BatchDev& b, const pgs_anchor_ptrs& A, const pgs_mlp_ptrs& W,
                                 const uint32_t* rows, const long long* n_rows, long long cap, const float* grad,
                                 const pgs_param_grad_ptrs& out, float* sc_dZ, float* sc_H, float* sc_dH, float* sc_X,
                                 uint32_t* err, cudaStream_t st);
// round_colour_h: the colour rows of dW2 take BF16-rounded H (the one-pass colour heads of PGS_DECODE_BF16)
void launch_mlp_wgrad(const float* dZ, const float* H, const float* dH, const float* X, const long long* n_rows,
                      long long cap, int in_dim, bool round_colour_h, float* partials, int nb,
                      const pgs_param_grad_ptrs& out, cudaStream_t st);

}  // namespace pgs
