// C ABI of libpgs: scene workspace and the launch sequence of the training
// step (see include/pgs.h for the contract of every entry point).
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

using namespace pgs;

namespace {

thread_local std::string g_last_error;

// autotuner choices per workload signature, process-wide
std::mutex g_tune_mu;
std::map<std::string, pgs_tune_entry> g_tune_cache;

pgs_status fail(pgs_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define PGS_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(PGS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

constexpr uint32_t kDefaultSpinLimit = 1u << 20;

__global__ void k_set_i64(long long* p, long long v) { *p = v; }
__global__ void k_iota(uint32_t* p, const long long* d_n) {
  const long long n = *d_n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = (uint32_t)i;
}
__global__ void k_zero_f4(float4* p, const long long* d_n, long long mult) {
  const long long n = *d_n * mult;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}
// rows = min(total, cap) (flag on overflow); G = 10 rows
__global__ void k_rows_total(const unsigned long long* total, long long cap, long long* d_rows, long long* d_g,
                             uint32_t* err) {
  const unsigned long long t = *total;
  if (t > (unsigned long long)cap) set_flag(err, kFlagCapacity);
  const long long r = (long long)min(t, (unsigned long long)cap);
  *d_rows = r;
  *d_g = r * kNOff;
}

template <typename T>
cudaError_t dmalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

}  // namespace

namespace pgs {
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace launch_cache {
std::mutex mu;
std::map<std::tuple<int, const void*, int, size_t>, int> occ;
std::map<int, int> sms;
}  // namespace launch_cache

int resident_ctas_per_sm(const void* kernel, int threads, size_t smem, int carveout) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  const auto key = std::make_tuple(dev, kernel, threads, smem);
  std::lock_guard<std::mutex> lk(launch_cache::mu);
  auto it = launch_cache::occ.find(key);
  if (it != launch_cache::occ.end()) return it->second;
  if (carveout >= 0) cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  launch_cache::occ[key] = per_sm;
  return per_sm;
}

int prepare_smem_kernel(const void* kernel, int threads, size_t smem) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  const auto key = std::make_tuple(dev, kernel, threads, smem);
  std::lock_guard<std::mutex> lk(launch_cache::mu);
  auto it = launch_cache::occ.find(key);
  if (it != launch_cache::occ.end()) return it->second;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  launch_cache::occ[key] = per_sm;
  return per_sm;
}

int device_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lk(launch_cache::mu);
  auto it = launch_cache::sms.find(dev);
  if (it != launch_cache::sms.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  launch_cache::sms[dev] = n;
  return n;
}
}  // namespace pgs

struct pgs_scene {
  pgs_scene_desc d{};
  int device = 0, num_sms = 148;
  bool bound = false;
  pgs_explicit_ptrs ex{};
  pgs_anchor_ptrs an{};
  pgs_mlp_ptrs mlp{};
  long long cap_g = 0, cap_rows = 0, cap_pairs = 0, max_tiles = 0, n_cull = 0;
  float4* rec = nullptr;
  float* grad_rec = nullptr;
  uint32_t *counts = nullptr, *keys_a = nullptr, *keys_b = nullptr, *gid_a = nullptr, *gid_b = nullptr;
  uint32_t* offs = nullptr;
  uint32_t *ptile_a = nullptr, *ptile_b = nullptr, *pg_a = nullptr, *pg_b = nullptr;
  uint2* ranges = nullptr;
  uint32_t *order_k = nullptr, *order_v = nullptr, *order_kb = nullptr, *order_vb = nullptr;  // tile queue
  uint32_t* queue_ctr = nullptr;         // [0] forward, [1] backward
  float *prior_partials = nullptr, *prior_means = nullptr;   // enhanced depth prior fit
  void* ncc_scratch = nullptr;                                // NCC per-pair counts, means, relative poses
  float* ncc_luma = nullptr;                                  // NCC: luma of the paired views [max_pixels]
  uint32_t *cull_flags = nullptr, *cull_offs = nullptr, *rows = nullptr;
  float *sc_dZ = nullptr, *sc_H = nullptr, *sc_dH = nullptr, *sc_X = nullptr, *wg_partials = nullptr;
  int wg_blocks = 0;
  long long* d_cnt = nullptr;            // [0] rows, [1] G, [2] P, [3] cull items, [4] tiles
  unsigned long long* d_tot = nullptr;   // [0] cull total, [1] pair total
  unsigned long long* scan_sums = nullptr;
  void* sort_mem = nullptr;
  SortScratch ss{};
  uint32_t* d_flags = nullptr;
  uint32_t* loss_counts = nullptr;
  float* loss_partials = nullptr;
  BatchDev batch{};
  bool have_batch = false;
  uint32_t spin_limit = kDefaultSpinLimit;
  uint32_t hold_tile = kNoHoldTile;   // failure-path test hook (pgs_scene_set_wait_limits)
  long long launches = 0;       // kernels enqueued since create
  bool prof = false;
  cudaEvent_t ev[PGS_N_STAGES][2] = {};
  bool ev_used[PGS_N_STAGES] = {};
};

namespace {
// stage brackets: CUDA events on the launching stream (external event nodes when captured)
// NVTX range names of the stages (pgs_stage order)
const char* const kStageRange[PGS_N_STAGES] = {"pgs:project", "pgs:depth_sort", "pgs:bin", "pgs:tile_sort",
                                               "pgs:blend_fwd", "pgs:loss", "pgs:blend_bwd", "pgs:project_bwd",
                                               "pgs:wgrad", "pgs:prior", "pgs:ncc", "pgs:tsdf"};

void prof_mark(pgs_scene* s, int stage, int which, cudaStream_t st) {
  if (!s->prof) return;
  if (which == 0) nvtxRangePushA(kStageRange[stage]);
  else nvtxRangePop();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  cudaEventRecordWithFlags(s->ev[stage][which], st, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0);
  s->ev_used[stage] = true;
}
}  // namespace

extern "C" {

const char* pgs_last_error(void) { return g_last_error.c_str(); }

int pgs_checked_build(void) { return kChecked ? 1 : 0; }

const char* pgs_status_string(pgs_status s) {
  switch (s) {
    case PGS_OK: return "ok";
    case PGS_ERR_INVALID_ARG: return "invalid argument";
    case PGS_ERR_CAPACITY: return "capacity exceeded";
    case PGS_ERR_TIMEOUT: return "bounded wait timed out";
    case PGS_ERR_NONFINITE: return "non-finite value";
    case PGS_ERR_CUDA: return "CUDA error";
    case PGS_ERR_UNSUPPORTED: return "unsupported";
    case PGS_ERR_BOUNDS: return "index out of bounds (checked build)";
    default: return "unknown status";
  }
}

void pgs_default_params(pgs_render_params* p) {
  if (!p) return;
  p->near_plane = 0.01f;
  p->dilation = 0.3f;
  p->alpha_min = 1.f / 255.f;
  p->alpha_max = 0.99f;
  p->t_min = 1e-4f;
  p->jclamp = 1.3f;
  p->tile_pad = 1e-3f;
  p->lod_d0 = 1e9f;
  p->n_levels = 1;
  p->bg = 0.f;
  p->tile_w = 16;
  p->tile_h = 16;
  p->decode_precision = PGS_DECODE_FP32;
  p->in_dim = 35;
  p->blend_batch = 256;
}

void pgs_scene_destroy(pgs_scene* s) {
  if (!s) return;
  void* ps[] = {s->rec, s->grad_rec, s->counts, s->keys_a, s->keys_b, s->gid_a, s->gid_b, s->offs, s->ptile_a,
                s->ptile_b, s->pg_a, s->pg_b, s->ranges, s->cull_flags, s->cull_offs, s->rows, s->sc_dZ, s->sc_H,
                s->sc_dH, s->sc_X, s->wg_partials, s->d_cnt, s->d_tot, s->scan_sums, s->sort_mem, s->d_flags,
                s->loss_counts, s->loss_partials, s->order_k, s->order_v, s->order_kb, s->order_vb,
                s->queue_ctr, s->prior_partials, s->prior_means, s->ncc_scratch, s->ncc_luma};
  for (void* p : ps)
    if (p) cudaFree(p);
  for (auto& e : s->ev)
    for (cudaEvent_t x : e)
      if (x) cudaEventDestroy(x);
  delete s;
}

pgs_status pgs_scene_create(const pgs_scene_desc* desc, pgs_scene** out) {
  if (!desc || !out) return fail(PGS_ERR_INVALID_ARG, "null descriptor or output");
  *out = nullptr;
  const pgs_scene_desc& d = *desc;
  const pgs_render_params& p = d.params;
  if (d.mode != PGS_MODE_EXPLICIT && d.mode != PGS_MODE_ANCHOR) return fail(PGS_ERR_INVALID_ARG, "mode %d", d.mode);
  if (d.n_primitives <= 0 || d.n_primitives >= (1ll << 27))
    return fail(PGS_ERR_INVALID_ARG, "n_primitives %lld", (long long)d.n_primitives);
  if (d.max_views <= 0 || d.max_views > PGS_MAX_VIEWS) return fail(PGS_ERR_INVALID_ARG, "max_views %d", d.max_views);
  if (d.max_pixels <= 0) return fail(PGS_ERR_INVALID_ARG, "max_pixels");
  if (d.capacity_pairs <= 0 || d.capacity_pairs >= (1ll << 30))
    return fail(PGS_ERR_INVALID_ARG, "capacity_pairs must be in (0, 2^30)");
  if (d.mode == PGS_MODE_ANCHOR && (d.capacity_rows <= 0 || d.capacity_rows * PGS_N_OFFSETS >= (1ll << 31)))
    return fail(PGS_ERR_INVALID_ARG, "capacity_rows");
  const bool tile_ok = (p.tile_w == 16 && p.tile_h == 16) || (p.tile_w == 8 && p.tile_h == 32) ||
                       (p.tile_w == 32 && p.tile_h == 8);
  if (!tile_ok) return fail(PGS_ERR_INVALID_ARG, "tile shape %dx%d (16x16, 8x32, 32x8)", p.tile_w, p.tile_h);
  if (p.in_dim != 35 && p.in_dim != 36) return fail(PGS_ERR_INVALID_ARG, "in_dim %d (35 or 36)", p.in_dim);
  if (p.blend_batch != 128 && p.blend_batch != 256 && p.blend_batch != 512)
    return fail(PGS_ERR_INVALID_ARG, "blend_batch %d (128, 256 or 512)", p.blend_batch);
  if (p.n_levels < 1 || p.n_levels > 16) return fail(PGS_ERR_INVALID_ARG, "n_levels %d", p.n_levels);
  if (!(p.alpha_min > 0.f && p.alpha_min < p.alpha_max && p.alpha_max < 1.f && p.t_min > 0.f && p.near_plane > 0.f))
    return fail(PGS_ERR_INVALID_ARG, "render thresholds out of range");
  if (p.decode_precision != PGS_DECODE_FP32 && p.decode_precision != PGS_DECODE_BF16 &&
      p.decode_precision != PGS_DECODE_BF16_1PASS)
    return fail(PGS_ERR_INVALID_ARG, "decode_precision");

  pgs_scene* s = new pgs_scene();
  s->d = d;
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
  const long long N = d.n_primitives;
  s->cap_rows = d.mode == PGS_MODE_ANCHOR ? d.capacity_rows : 0;
  s->cap_g = d.mode == PGS_MODE_EXPLICIT ? N * d.max_views : s->cap_rows * PGS_N_OFFSETS;
  if (s->cap_g >= (1ll << 31)) { delete s; return fail(PGS_ERR_INVALID_ARG, "Gaussian-view capacity too large"); }
  s->cap_pairs = d.capacity_pairs;
  s->max_tiles = d.max_pixels / 64 + (long long)d.max_views * 1024;
  s->n_cull = d.mode == PGS_MODE_ANCHOR ? N * d.max_views : 0;
  const long long sort_n = std::max(std::max(s->cap_g, s->cap_pairs), s->max_tiles);
  s->ss = sort_scratch_layout(nullptr, sort_n, 9);
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, n) if (e == cudaSuccess) e = dmalloc(&(ptr), (size_t)(n))
  ALLOC(s->rec, s->cap_g * kRecF4);
  ALLOC(s->grad_rec, s->cap_g * 16);
  ALLOC(s->counts, s->cap_g);
  ALLOC(s->keys_a, s->cap_g);
  ALLOC(s->keys_b, s->cap_g);
  ALLOC(s->gid_a, s->cap_g);
  ALLOC(s->gid_b, s->cap_g);
  ALLOC(s->offs, s->cap_g);
  ALLOC(s->ptile_a, s->cap_pairs);
  ALLOC(s->ptile_b, s->cap_pairs);
  ALLOC(s->pg_a, s->cap_pairs);
  ALLOC(s->pg_b, s->cap_pairs);
  ALLOC(s->ranges, s->max_tiles);
  ALLOC(s->order_k, s->max_tiles);
  ALLOC(s->order_v, s->max_tiles);
  ALLOC(s->order_kb, s->max_tiles);
  ALLOC(s->order_vb, s->max_tiles);
  ALLOC(s->queue_ctr, 2);
  ALLOC(s->prior_partials, (long long)kMaxViews * kPriorBlocks * 3);
  ALLOC(s->prior_means, (long long)kMaxViews * 4);
  if (e == cudaSuccess) e = cudaMalloc(&s->ncc_scratch, ncc_scratch_bytes());
  ALLOC(s->ncc_luma, d.max_pixels);
  ALLOC(s->d_cnt, 8);
  ALLOC(s->d_tot, 4);
  ALLOC(s->scan_sums, kScanBlocks);
  ALLOC(s->d_flags, 4);
  ALLOC(s->loss_counts, kMaxViews * 2);
  ALLOC(s->loss_partials, kLossBlocks * 3);
  if (e == cudaSuccess) e = cudaMalloc(&s->sort_mem, s->ss.bytes);
  if (d.mode == PGS_MODE_ANCHOR) {
    ALLOC(s->cull_flags, s->n_cull);
    ALLOC(s->cull_offs, s->n_cull);
    ALLOC(s->rows, s->cap_rows);
    ALLOC(s->sc_dZ, sc_rows(s->cap_rows) * kOut);
    ALLOC(s->sc_H, sc_rows(s->cap_rows) * kHidden);
    ALLOC(s->sc_dH, sc_rows(s->cap_rows) * kHidden);
    ALLOC(s->sc_X, sc_rows(s->cap_rows) * kMaxIn);
    s->wg_blocks = 2 * s->num_sms;
    ALLOC(s->wg_partials, (long long)s->wg_blocks * mlp_wgrad_outputs(kMaxIn));
  }
#undef ALLOC
  if (e != cudaSuccess) {
    pgs_scene_destroy(s);
    return fail(PGS_ERR_CUDA, "workspace allocation: %s", cudaGetErrorString(e));
  }
  s->ss = sort_scratch_layout(s->sort_mem, sort_n, 9);
  e = cudaMemset(s->d_flags, 0, 4 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(s->d_cnt, 0, 8 * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(s->ss.err, 0, sizeof(uint32_t));
  if (e != cudaSuccess) {
    pgs_scene_destroy(s);
    return fail(PGS_ERR_CUDA, "workspace init: %s", cudaGetErrorString(e));
  }
  *out = s;
  return PGS_OK;
}

pgs_status pgs_scene_bind_explicit(pgs_scene* s, const pgs_explicit_ptrs* p) {
  if (!s || !p) return fail(PGS_ERR_INVALID_ARG, "null scene or pointers");
  if (s->d.mode != PGS_MODE_EXPLICIT) return fail(PGS_ERR_INVALID_ARG, "scene is not in explicit mode");
  if (!p->means || !p->log_scales || !p->quats || !p->opacity_logits || !p->colors)
    return fail(PGS_ERR_INVALID_ARG, "null parameter pointer");
  s->ex = *p;
  s->bound = true;
  return PGS_OK;
}

pgs_status pgs_scene_bind_anchors(pgs_scene* s, const pgs_anchor_ptrs* a, const pgs_mlp_ptrs* w) {
  if (!s || !a || !w) return fail(PGS_ERR_INVALID_ARG, "null scene or pointers");
  if (s->d.mode != PGS_MODE_ANCHOR) return fail(PGS_ERR_INVALID_ARG, "scene is not in anchor mode");
  if (!a->x || !a->level || !a->log_l || !a->offsets || !a->feat || !w->W1 || !w->b1 || !w->W2 || !w->b2)
    return fail(PGS_ERR_INVALID_ARG, "null parameter pointer");
  if ((reinterpret_cast<uintptr_t>(a->feat) & 15) != 0) return fail(PGS_ERR_INVALID_ARG, "feat must be 16-byte aligned");
  s->an = *a;
  s->mlp = *w;
  s->bound = true;
  return PGS_OK;
}

}  // extern "C"

namespace {

pgs_status build_batch(pgs_scene* s, const pgs_camera* cams, int n_views, BatchDev& b) {
  if (!cams || n_views <= 0 || n_views > s->d.max_views)
    return fail(PGS_ERR_INVALID_ARG, "n_views %d (max %d)", n_views, s->d.max_views);
  std::memset(&b, 0, sizeof(b));
  const pgs_render_params& p = s->d.params;
  b.p.near_plane = p.near_plane; b.p.dilation = p.dilation; b.p.alpha_min = p.alpha_min; b.p.alpha_max = p.alpha_max;
  b.p.t_min = p.t_min; b.p.jclamp = p.jclamp; b.p.tile_pad = p.tile_pad; b.p.lod_d0 = p.lod_d0; b.p.bg = p.bg;
  b.p.n_levels = p.n_levels; b.p.tile_w = p.tile_w; b.p.tile_h = p.tile_h; b.p.in_dim = p.in_dim;
  b.p.blend_batch = p.blend_batch;
  b.p.decode = p.decode_precision;
  b.n_views = n_views;
  long long pix = 0;
  long long tiles = 0;
  for (int i = 0; i < n_views; ++i) {
    const pgs_camera& c = cams[i];
    ViewDev& v = b.v[i];
    if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384 || !(c.fx > 0.f) || !(c.fy > 0.f))
      return fail(PGS_ERR_INVALID_ARG, "camera %d: bad size or focal length", i);
    std::memcpy(v.R, c.R, sizeof(v.R));
    std::memcpy(v.t, c.t, sizeof(v.t));
    v.fx = c.fx; v.fy = c.fy; v.cx = c.cx; v.cy = c.cy;
    v.W = c.width; v.H = c.height;
    for (int k = 0; k < 3; ++k)   // centre = -R^T t
      v.center[k] = (float)(-((double)c.R[k] * c.t[0] + (double)c.R[3 + k] * c.t[1] + (double)c.R[6 + k] * c.t[2]));
    v.lim_x = p.jclamp * 0.5f * (float)c.width / c.fx;
    v.lim_y = p.jclamp * 0.5f * (float)c.height / c.fy;
    v.tiles_x = (c.width + p.tile_w - 1) / p.tile_w;
    v.tiles_y = (c.height + p.tile_h - 1) / p.tile_h;
    v.tile_base = (int)tiles;
    v.pix_off = pix;
    tiles += (long long)v.tiles_x * v.tiles_y;
    pix += (long long)c.width * c.height;
  }
  if (pix > s->d.max_pixels)
    return fail(PGS_ERR_INVALID_ARG, "batch has %lld pixels > max_pixels %lld", pix, (long long)s->d.max_pixels);
  if (tiles > s->max_tiles) return fail(PGS_ERR_INVALID_ARG, "batch has %lld tiles > %lld", tiles, s->max_tiles);
  b.total_tiles = (int)tiles;
  b.total_pixels = pix;
  b.cap_pairs = s->cap_pairs;
  b.cap_g = s->cap_g;
  b.flags = s->d_flags;
  return PGS_OK;
}

int tile_bits(long long tiles) {
  int bits = 1;
  while ((1ll << bits) < tiles) ++bits;
  return bits;
}

int grid_for(long long n, int block, int num_sms, int per_sm = 8) {
  long long g = (n + block - 1) / block;
  g = std::min<long long>(g, (long long)num_sms * per_sm);
  return (int)std::max<long long>(g, 1);
}

// cull + compact + decode/project (anchor) or project (explicit); leaves d_cnt[1] = G
pgs_status run_project(pgs_scene* s, const BatchDev& b, DecodeOut dec, bool project, cudaStream_t st) {
  const int ns = s->num_sms;
  prof_mark(s, PGS_STAGE_PROJECT, 0, st);
  if (s->d.mode == PGS_MODE_EXPLICIT) {
    const long long G = s->d.n_primitives * b.n_views;
    k_set_i64<<<1, 1, 0, st>>>(s->d_cnt + 1, G);
    k_project_explicit<<<grid_for(G, 256, ns), 256, 0, st>>>(b, s->ex, s->d.n_primitives, s->rec, s->counts, s->keys_a,
                                                             s->d_flags);
    s->launches += 2;
  } else {
    const long long Na = s->d.n_primitives;
    const long long tot = Na * b.n_views;
    k_anchor_cull<<<grid_for(tot, 256, ns), 256, 0, st>>>(b, s->an, Na, s->cull_flags);
    k_set_i64<<<1, 1, 0, st>>>(s->d_cnt + 3, tot);
    launch_exclusive_scan(s->cull_flags, nullptr, s->cull_offs, s->d_tot, s->d_cnt + 3, s->scan_sums, st);
    k_compact_rows<<<grid_for(tot, 256, ns), 256, 0, st>>>(s->cull_flags, s->cull_offs, tot, Na, s->rows, s->cap_rows,
                                                          s->d_flags);
    k_rows_total<<<1, 1, 0, st>>>(s->d_tot, s->cap_rows, s->d_cnt, s->d_cnt + 1, s->d_flags);
    const int prec = s->d.params.decode_precision;
    if (prec == PGS_DECODE_BF16 || prec == PGS_DECODE_BF16_1PASS) {
      // the decoded outputs pass through the decoder-backward row scratch (free until pgs_backward)
      PGS_CUDA(launch_decode_project_tc(prec == PGS_DECODE_BF16, b, s->an, s->mlp, s->rows, s->d_cnt, s->cap_rows,
                                        s->sc_dZ, project ? s->rec : nullptr, s->counts, s->keys_a, dec, s->d_flags,
                                        st));
    } else {
      k_decode_project<<<ns * 4, 256, 0, st>>>(b, s->an, s->mlp, s->rows, s->d_cnt, s->cap_rows,
                                              project ? s->rec : nullptr, s->counts, s->keys_a, dec, s->d_flags);
    }
    s->launches += 5 + kScanLaunches + ((prec == PGS_DECODE_BF16 || prec == PGS_DECODE_BF16_1PASS) ? 1 : 0);
  }
  prof_mark(s, PGS_STAGE_PROJECT, 1, st);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

}  // namespace

extern "C" {

pgs_status pgs_decode_anchors(pgs_scene* s, const pgs_camera* cams, int n_views, uint32_t* d_rows, float* d_mu,
                              float* d_opacity, float* d_color, float* d_scale, float* d_quat, int64_t* d_n_rows,
                              cudaStream_t stream) {
  if (!s || !s->bound) return fail(PGS_ERR_INVALID_ARG, "scene not bound");
  if (s->d.mode != PGS_MODE_ANCHOR) return fail(PGS_ERR_INVALID_ARG, "pgs_decode_anchors needs anchor mode");
  if (!d_rows || !d_mu || !d_opacity || !d_color || !d_scale || !d_quat || !d_n_rows)
    return fail(PGS_ERR_INVALID_ARG, "null output pointer");
  BatchDev b;
  pgs_status r = build_batch(s, cams, n_views, b);
  if (r) return r;
  DecodeOut dec{d_mu, d_opacity, d_color, d_scale, d_quat};
  r = run_project(s, b, dec, false, stream);
  if (r) return r;
  PGS_CUDA(cudaMemcpyAsync(d_rows, s->rows, (size_t)s->cap_rows * sizeof(uint32_t), cudaMemcpyDeviceToDevice, stream));
  PGS_CUDA(cudaMemcpyAsync(d_n_rows, s->d_cnt, sizeof(long long), cudaMemcpyDeviceToDevice, stream));
  return PGS_OK;
}

pgs_status pgs_render_batch(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* out,
                            cudaStream_t st) {
  if (!s || !s->bound) return fail(PGS_ERR_INVALID_ARG, "scene not bound");
  if (!out || !out->rgb || !out->depth || !out->normal || !out->dist || !out->t_final || !out->last)
    return fail(PGS_ERR_INVALID_ARG, "null image pointer (rgb, depth, normal, dist, t_final, last are required)");
  BatchDev b;
  pgs_status r = build_batch(s, cams, n_views, b);
  if (r) return r;
  const int ns = s->num_sms;
  r = run_project(s, b, DecodeOut{}, true, st);
  if (r) return r;
  long long* d_G = s->d_cnt + 1;
  long long* d_P = s->d_cnt + 2;
  int nl = 0;
  // depth order of the Gaussian-views (stable: ties keep index order)
  prof_mark(s, PGS_STAGE_DEPTH_SORT, 0, st);
  k_iota<<<ns * 4, 256, 0, st>>>(s->gid_a, d_G);
  PGS_CUDA(launch_sort_pairs(s->keys_a, s->gid_a, s->keys_b, s->gid_b, d_G, s->cap_g, 0, 32, s->ss, s->d_flags,
                             s->spin_limit, s->hold_tile, ns, st, &nl));
  // a look-back wait that ran out leaves the order unspecified: fall back to index order (valid ids only)
  k_sort_timeout_guard<<<ns * 2, 256, 0, st>>>(s->d_flags, s->d_cnt + 1, s->cap_g, s->gid_a);
  s->launches += 2 + nl;
  prof_mark(s, PGS_STAGE_DEPTH_SORT, 1, st);
  // pair offsets in depth order, then emission
  prof_mark(s, PGS_STAGE_BIN, 0, st);
  launch_exclusive_scan(s->counts, s->gid_a, s->offs, s->d_tot + 1, d_G, s->scan_sums, st);
  k_pairs_total<<<1, 1, 0, st>>>(s->d_tot + 1, s->cap_pairs, d_P, s->d_flags);
  k_emit_pairs<<<ns * 16, 128, 0, st>>>(b, s->rec, s->counts, s->gid_a, s->offs, d_G, s->cap_pairs, s->d.mode,
                                       s->d.n_primitives, s->rows, s->ptile_a, s->pg_a, s->d_flags);
  s->launches += kScanLaunches + 2;
  prof_mark(s, PGS_STAGE_BIN, 1, st);
  // stable sort of the pairs by tile, then per-tile ranges
  prof_mark(s, PGS_STAGE_TILE_SORT, 0, st);
  PGS_CUDA(launch_sort_pairs(s->ptile_a, s->pg_a, s->ptile_b, s->pg_b, d_P, s->cap_pairs, 0, tile_bits(b.total_tiles),
                             s->ss, s->d_flags, s->spin_limit, s->hold_tile, ns, st, &nl));
  k_sort_timeout_guard<<<1, 32, 0, st>>>(s->d_flags, d_P, s->cap_pairs, nullptr);   // ran out: no pairs
  PGS_CUDA(cudaMemsetAsync(s->ranges, 0, (size_t)b.total_tiles * sizeof(uint2), st));
  k_tile_ranges<<<ns * 8, 256, 0, st>>>(s->ptile_a, d_P, s->ranges, b.total_tiles, s->d_flags);
  s->launches += nl + 2;
  // queue order for the persistent blend kernels: longest tile lists first (16-bit keys, two passes)
  constexpr int kTileOrderBits = 16;
  k_set_i64<<<1, 1, 0, st>>>(s->d_cnt + 4, b.total_tiles);
  k_tile_order_keys<<<ns * 2, 256, 0, st>>>(s->ranges, b.total_tiles, s->order_k, s->order_v);
  PGS_CUDA(launch_sort_pairs(s->order_k, s->order_v, s->order_kb, s->order_vb, s->d_cnt + 4, s->max_tiles, 0, kTileOrderBits,
                             s->ss, s->d_flags, s->spin_limit, s->hold_tile, ns, st, &nl));
  k_sort_timeout_guard<<<ns, 256, 0, st>>>(s->d_flags, s->d_cnt + 4, s->max_tiles, s->order_v);  // ran out: tile order
  s->launches += 3 + nl;
  prof_mark(s, PGS_STAGE_TILE_SORT, 1, st);
  prof_mark(s, PGS_STAGE_BLEND_FWD, 0, st);
  PGS_CUDA(cudaMemsetAsync(s->queue_ctr, 0, 2 * sizeof(uint32_t), st));
  if (!launch_blend_fwd(b, s->rec, s->pg_a, s->ranges, *out, s->order_v, s->queue_ctr, st))
    return fail(PGS_ERR_UNSUPPORTED, "tile shape");
  s->launches += 1;
  prof_mark(s, PGS_STAGE_BLEND_FWD, 1, st);
  PGS_CUDA(cudaGetLastError());
  s->batch = b;
  s->have_batch = true;
  return PGS_OK;
}

pgs_status pgs_loss_grad(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* img,
                         const pgs_target_ptrs* tgt, const pgs_loss_params* lp, float* d_loss,
                         const pgs_image_grad_ptrs* grad, cudaStream_t st) {
  if (!s || !img || !tgt || !lp || !d_loss || !grad) return fail(PGS_ERR_INVALID_ARG, "null argument");
  if (!img->rgb || !img->depth || !img->normal || !tgt->rgb || !tgt->prior || !tgt->mask || !grad->rgb ||
      !grad->depth || !grad->normal)
    return fail(PGS_ERR_INVALID_ARG, "null image, target or gradient pointer");
  BatchDev b;
  pgs_status r = build_batch(s, cams, n_views, b);
  if (r) return r;
  prof_mark(s, PGS_STAGE_LOSS, 0, st);
  launch_loss(b, *img, *tgt, *lp, d_loss, *grad, s->loss_counts, s->loss_partials, s->d_flags, st);
  s->launches += kLossLaunches;
  prof_mark(s, PGS_STAGE_LOSS, 1, st);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

pgs_status pgs_backward(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* img,
                        const pgs_image_grad_ptrs* grad, const pgs_param_grad_ptrs* pg, cudaStream_t st) {
  if (!s || !s->bound || !img || !grad || !pg) return fail(PGS_ERR_INVALID_ARG, "null argument or scene not bound");
  if (!s->have_batch) return fail(PGS_ERR_INVALID_ARG, "pgs_backward before any pgs_render_batch");
  if (!img->normal || !img->dist || !img->t_final || !img->last || !grad->rgb || !grad->depth || !grad->normal)
    return fail(PGS_ERR_INVALID_ARG, "null image or gradient pointer");
  BatchDev b;
  pgs_status r = build_batch(s, cams, n_views, b);
  if (r) return r;
  if (b.total_tiles != s->batch.total_tiles || b.total_pixels != s->batch.total_pixels)
    return fail(PGS_ERR_INVALID_ARG, "cameras differ from the last pgs_render_batch");
  const int ns = s->num_sms;
  const long long* d_G = s->d_cnt + 1;
  prof_mark(s, PGS_STAGE_BLEND_BWD, 0, st);
  k_zero_f4<<<ns * 4, 256, 0, st>>>(reinterpret_cast<float4*>(s->grad_rec), d_G, 4);
  PGS_CUDA(cudaMemsetAsync(s->queue_ctr + 1, 0, sizeof(uint32_t), st));
  if (!launch_blend_bwd(b, s->rec, s->pg_a, s->ranges, *img, *grad, s->grad_rec, s->order_v, s->queue_ctr + 1, st))
    return fail(PGS_ERR_UNSUPPORTED, "tile shape");
  s->launches += 2;
  prof_mark(s, PGS_STAGE_BLEND_BWD, 1, st);
  prof_mark(s, PGS_STAGE_PROJECT_BWD, 0, st);
  if (s->d.mode == PGS_MODE_EXPLICIT) {
    const long long G = s->d.n_primitives * b.n_views;
    k_project_bwd_explicit<<<grid_for(G, 128, ns, 16), 128, 0, st>>>(b, s->ex, s->d.n_primitives, s->grad_rec, *pg,
                                                                     s->d_flags);
    s->launches += 1;
    prof_mark(s, PGS_STAGE_PROJECT_BWD, 1, st);
  } else if (s->d.params.decode_precision == PGS_DECODE_BF16) {
    // the tensor-core decoder's backward on the tensor cores
    PGS_CUDA(launch_decode_bwd_tc(b, s->an, s->mlp, s->rows, s->d_cnt, s->cap_rows, s->grad_rec, *pg, s->sc_dZ,
                                  s->sc_H, s->sc_dH, s->sc_X, s->d_flags, st));
    s->launches += 1;
    prof_mark(s, PGS_STAGE_PROJECT_BWD, 1, st);
    prof_mark(s, PGS_STAGE_WGRAD, 0, st);
    PGS_CUDA(launch_mlp_wgrad_tc(s->sc_dZ, s->sc_H, s->sc_dH, s->sc_X, s->d_cnt, s->cap_rows, s->d.params.in_dim,
                                 s->wg_partials, s->wg_blocks, *pg, s->d_flags, st));
    s->launches += 2;
    prof_mark(s, PGS_STAGE_WGRAD, 1, st);
  } else {
    k_decode_bwd<<<ns * 4, 128, 0, st>>>(b, s->an, s->mlp, s->rows, s->d_cnt, s->cap_rows, s->grad_rec, *pg, s->sc_dZ,
                                        s->sc_H, s->sc_dH, s->sc_X, s->d_flags);
    s->launches += 1;
    prof_mark(s, PGS_STAGE_PROJECT_BWD, 1, st);
    prof_mark(s, PGS_STAGE_WGRAD, 0, st);
    launch_mlp_wgrad(s->sc_dZ, s->sc_H, s->sc_dH, s->sc_X, s->d_cnt, s->cap_rows, s->d.params.in_dim,
                     s->d.params.decode_precision == PGS_DECODE_BF16, s->wg_partials, s->wg_blocks, *pg, st);
    s->launches += kWgradLaunches;
    prof_mark(s, PGS_STAGE_WGRAD, 1, st);
  }
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

pgs_status pgs_scene_set_wait_limits(pgs_scene* s, uint32_t spin_limit, uint32_t withhold_tile) {
  if (!s) return fail(PGS_ERR_INVALID_ARG, "null scene");
  s->spin_limit = spin_limit ? spin_limit : kDefaultSpinLimit;
  s->hold_tile = withhold_tile;
  return PGS_OK;
}

pgs_status pgs_set_profiling(pgs_scene* s, int enable) {
  if (!s) return fail(PGS_ERR_INVALID_ARG, "null scene");
  if (enable && !s->ev[0][0]) {
    for (auto& e : s->ev)
      for (cudaEvent_t& x : e) PGS_CUDA(cudaEventCreate(&x));
  }
  s->prof = enable != 0;
  for (bool& u : s->ev_used) u = false;
  return PGS_OK;
}

pgs_status pgs_get_stage_times(pgs_scene* s, float* ms, int n) {
  if (!s || !ms || n <= 0) return fail(PGS_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < n && k < PGS_N_STAGES; ++k) {
    ms[k] = -1.f;
    if (!s->ev_used[k]) continue;
    PGS_CUDA(cudaEventSynchronize(s->ev[k][1]));
    PGS_CUDA(cudaEventElapsedTime(&ms[k], s->ev[k][0], s->ev[k][1]));
  }
  return PGS_OK;
}

pgs_status pgs_filter_depth_prior(pgs_scene* s, const pgs_camera* cams, int n_views, const float* d_pseudo,
                                  const float* d_points, int64_t n_points, const pgs_prior_params* pp,
                                  float* d_prior_out, float* d_mask_out, float* d_scale_shift, float* d_err_out,
                                  cudaStream_t st) {
  if (!s || !pp || !d_pseudo || !d_prior_out || !d_mask_out || !d_scale_shift)
    return fail(PGS_ERR_INVALID_ARG, "null argument");
  if (n_points < 0 || (n_points > 0 && !d_points)) return fail(PGS_ERR_INVALID_ARG, "points");
  if (!(pp->tau_d > 0.f) || pp->k_neighbors < 1 || pp->k_neighbors > kPriorMaxK)
    return fail(PGS_ERR_INVALID_ARG, "tau_d %g, k_neighbors %d (1..%d)", pp->tau_d, pp->k_neighbors, kPriorMaxK);
  BatchDev b;
  pgs_status r = build_batch(s, cams, n_views, b);
  if (r) return r;
  // the k nearest other views by camera centre (ties by index)
  PriorArgs pa;
  pa.k = std::min(pp->k_neighbors, n_views - 1);
  pa.tau_d = pp->tau_d;
  for (int a = 0; a < kMaxViews; ++a)
    for (int i = 0; i < kPriorMaxK; ++i) pa.nbr[a][i] = -1;
  for (int a = 0; a < n_views; ++a) {
    std::vector<std::pair<double, int>> d;
    for (int c = 0; c < n_views; ++c) {
      if (c == a) continue;
      double q = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double e = (double)b.v[a].center[k] - (double)b.v[c].center[k];
        q += e * e;
      }
      d.emplace_back(q, c);
    }
    std::sort(d.begin(), d.end());
    for (int i = 0; i < pa.k; ++i) pa.nbr[a][i] = d[i].second;
  }
  prof_mark(s, PGS_STAGE_PRIOR, 0, st);
  launch_prior_filter(b, pa, d_pseudo, d_points, (long long)n_points, s->prior_partials, s->prior_means,
                      d_scale_shift, d_prior_out, d_mask_out, d_err_out, s->num_sms, st);
  s->launches += kPriorLaunches;
  prof_mark(s, PGS_STAGE_PRIOR, 1, st);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

pgs_status pgs_ncc_loss_grad(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* img,
                             const uint32_t* d_centers, int64_t n_per_pair, const pgs_ncc_params* np, float* d_ncc,
                             float* d_loss, const pgs_image_grad_ptrs* grad, cudaStream_t st) {
  if (!s || !img || !np || !d_loss || !grad) return fail(PGS_ERR_INVALID_ARG, "null argument");
  if (!img->rgb || !img->depth || !img->normal || !grad->rgb || (np->geometric && (!grad->depth || !grad->normal)))
    return fail(PGS_ERR_INVALID_ARG, "null image or gradient pointer");
  if (n_per_pair < 0 || n_per_pair > (int64_t(1) << 26)) return fail(PGS_ERR_INVALID_ARG, "n_per_pair %lld",
                                                                    (long long)n_per_pair);
  if (!(np->eps >= 0.f) || !std::isfinite(np->lambda_ncc)) return fail(PGS_ERR_INVALID_ARG, "eps or lambda_ncc");
  BatchDev b;
  pgs_status r = build_batch(s, cams, n_views, b);
  if (r) return r;
  const int n_pairs = n_views / 2;
  if (n_pairs > 0 && n_per_pair > 0 && (!d_centers || !d_ncc))
    return fail(PGS_ERR_INVALID_ARG, "null centres or NCC output");
  NccArgs a;
  a.lambda = np->lambda_ncc;
  a.eps = np->eps;
  a.geometric = np->geometric ? 1 : 0;
  prof_mark(s, PGS_STAGE_NCC, 0, st);
  PGS_CUDA(launch_ncc(b, a, d_centers, (long long)n_per_pair, n_pairs, img->rgb, img->depth, img->normal, d_ncc,
                      d_loss, grad->rgb, grad->depth, grad->normal, s->ncc_scratch, s->ncc_luma, s->num_sms, st));
  s->launches += (n_pairs > 0 && n_per_pair > 0) ? kNccLaunches : 0;
  prof_mark(s, PGS_STAGE_NCC, 1, st);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

pgs_status pgs_tsdf_integrate(pgs_scene* s, const pgs_camera* cams, int n_views, const float* d_depth,
                              const float* d_rgb, const pgs_tsdf_volume* vol, float* d_tsdf, float* d_weight,
                              float* d_color, cudaStream_t st) {
  if (!s || !vol || !d_depth || !d_tsdf || !d_weight) return fail(PGS_ERR_INVALID_ARG, "null argument");
  if ((d_rgb == nullptr) != (d_color == nullptr)) return fail(PGS_ERR_INVALID_ARG, "colour in and out go together");
  if (vol->dims[0] < 1 || vol->dims[1] < 1 || vol->dims[2] < 1 ||
      (long long)vol->dims[0] * vol->dims[1] * vol->dims[2] > (1ll << 34))
    return fail(PGS_ERR_INVALID_ARG, "dims %d x %d x %d", vol->dims[0], vol->dims[1], vol->dims[2]);
  if (!(vol->voxel > 0.f) || !(vol->trunc > 0.f) || !std::isfinite(vol->origin[0]) ||
      !std::isfinite(vol->origin[1]) || !std::isfinite(vol->origin[2]))
    return fail(PGS_ERR_INVALID_ARG, "voxel, trunc or origin");
  BatchDev b;
  pgs_status r = build_batch(s, cams, n_views, b);
  if (r) return r;
  TsdfArgs a;
  for (int k = 0; k < 3; ++k) {
    a.origin[k] = vol->origin[k];
    a.dims[k] = vol->dims[k];
  }
  a.voxel = vol->voxel;
  a.trunc = vol->trunc;
  // the tile-sort buffer ptile_b (sort scratch, free between renders) holds the interleaved maps when it is large
  // enough (16 B per pixel); otherwise the colour planes are read directly
  float4* pack = (d_rgb && s->cap_pairs * (long long)sizeof(uint32_t) >= b.total_pixels * (long long)sizeof(float4))
                     ? reinterpret_cast<float4*>(s->ptile_b)
                     : nullptr;
  prof_mark(s, PGS_STAGE_TSDF, 0, st);
  s->launches += launch_tsdf(b, a, d_depth, d_rgb, pack, d_tsdf, d_weight, d_color, s->num_sms, st);
  prof_mark(s, PGS_STAGE_TSDF, 1, st);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

pgs_status pgs_scene_get_params(const pgs_scene* s, pgs_render_params* out) {
  if (!s || !out) return fail(PGS_ERR_INVALID_ARG, "null argument");
  *out = s->d.params;
  return PGS_OK;
}

pgs_status pgs_autotune(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* img,
                        const pgs_image_grad_ptrs* grad, const pgs_param_grad_ptrs* pg, int reps,
                        pgs_tune_entry* entries, int max_entries, int* n_entries, cudaStream_t st) {
  if (n_entries) *n_entries = 0;
  if (!s || !cams || !img || !grad || !pg) return fail(PGS_ERR_INVALID_ARG, "null argument");
  if (n_views <= 0 || n_views > s->d.max_views) return fail(PGS_ERR_INVALID_ARG, "n_views %d", n_views);
  if (reps < 1 || reps > 100) return fail(PGS_ERR_INVALID_ARG, "reps %d (1..100)", reps);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  PGS_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(PGS_ERR_INVALID_ARG, "pgs_autotune during stream capture");
  // workload signature
  std::string key = std::to_string(s->device) + "/" + std::to_string(s->d.mode) + "/" +
                    std::to_string(s->d.n_primitives);
  for (int v = 0; v < n_views; ++v) key += "/" + std::to_string(cams[v].width) + "x" + std::to_string(cams[v].height);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      s->d.params.tile_w = it->second.tile_w;
      s->d.params.tile_h = it->second.tile_h;
      s->d.params.blend_batch = it->second.blend_batch;
      if (entries && max_entries > 0) {
        entries[0] = it->second;
        entries[0].ms = -1.f;
        if (n_entries) *n_entries = 1;
      }
      return PGS_OK;
    }
  }
  static const int shapes[3][2] = {{16, 16}, {8, 32}, {32, 8}};
  static const int batches[3] = {128, 256, 512};
  const pgs_render_params saved = s->d.params;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PGS_CUDA(cudaEventCreate(&e0));
  PGS_CUDA(cudaEventCreate(&e1));
  pgs_tune_entry best{saved.tile_w, saved.tile_h, saved.blend_batch, 3.4e38f};
  int n = 0;
  pgs_status r = PGS_OK;
  for (const auto& sh : shapes) {
    for (int nb : batches) {
      s->d.params.tile_w = sh[0];
      s->d.params.tile_h = sh[1];
      s->d.params.blend_batch = nb;
      std::vector<float> t;
      for (int k = 0; k <= reps && r == PGS_OK; ++k) {
        if (k > 0) cudaEventRecord(e0, st);
        r = pgs_render_batch(s, cams, n_views, img, st);
        if (r == PGS_OK) r = pgs_backward(s, cams, n_views, img, grad, pg, st);
        if (k > 0 && r == PGS_OK) {
          cudaEventRecord(e1, st);
          float ms = 0.f;
          if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            r = fail(PGS_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(cudaGetLastError()));
            break;
          }
          t.push_back(ms);
        }
      }
      if (r != PGS_OK) break;
      std::sort(t.begin(), t.end());
      const pgs_tune_entry e{sh[0], sh[1], nb, t[t.size() / 2]};
      if (entries && n < max_entries) entries[n] = e;
      ++n;
      if (e.ms < best.ms) best = e;
    }
    if (r != PGS_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != PGS_OK) {
    s->d.params = saved;
    return r;
  }
  if (n_entries) *n_entries = std::min(n, max_entries);
  s->d.params.tile_w = best.tile_w;
  s->d.params.tile_h = best.tile_h;
  s->d.params.blend_batch = best.blend_batch;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return PGS_OK;
}

pgs_status pgs_read_status(pgs_scene* s, cudaStream_t st) {
  if (!s) return fail(PGS_ERR_INVALID_ARG, "null scene");
  PGS_CUDA(cudaStreamSynchronize(st));
  uint32_t f = 0, e2 = 0;
  PGS_CUDA(cudaMemcpy(&f, s->d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  PGS_CUDA(cudaMemcpy(&e2, s->ss.err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  f |= e2;
  PGS_CUDA(cudaMemset(s->d_flags, 0, sizeof(uint32_t)));
  PGS_CUDA(cudaMemset(s->ss.err, 0, sizeof(uint32_t)));
  for (int c : {PGS_ERR_BOUNDS, PGS_ERR_CAPACITY, PGS_ERR_TIMEOUT, PGS_ERR_NONFINITE})
    if (f & (1u << c)) return fail(c, "device reported: %s", pgs_status_string(c));
  return PGS_OK;
}

pgs_status pgs_get_stats(pgs_scene* s, pgs_stats* out, cudaStream_t st) {
  if (!s || !out) return fail(PGS_ERR_INVALID_ARG, "null argument");
  PGS_CUDA(cudaStreamSynchronize(st));
  long long c[4];
  PGS_CUDA(cudaMemcpy(c, s->d_cnt, sizeof(c), cudaMemcpyDeviceToHost));
  uint32_t f = 0;
  PGS_CUDA(cudaMemcpy(&f, s->d_flags, sizeof(f), cudaMemcpyDeviceToHost));
  out->rows = s->d.mode == PGS_MODE_ANCHOR ? c[0] : 0;
  out->gaussian_views = c[1];
  out->pairs = c[2];
  out->tiles = s->have_batch ? s->batch.total_tiles : 0;
  out->pixels = s->have_batch ? s->batch.total_pixels : 0;
  out->flags = f;
  out->launches = s->launches;
  return PGS_OK;
}

pgs_status pgs_scene_buffer(pgs_scene* s, int which, void** d_ptr, int64_t* cap) {
  if (!s || !d_ptr || !cap) return fail(PGS_ERR_INVALID_ARG, "null argument");
  switch (which) {
    case 0: *d_ptr = s->rec; *cap = s->cap_g * 16; break;
    case 1: *d_ptr = s->counts; *cap = s->cap_g; break;
    case 2: *d_ptr = s->ptile_a; *cap = s->cap_pairs; break;
    case 3: *d_ptr = s->pg_a; *cap = s->cap_pairs; break;
    case 4: *d_ptr = s->ranges; *cap = s->max_tiles * 2; break;
    case 5: *d_ptr = s->gid_a; *cap = s->cap_g; break;
    case 6: *d_ptr = s->rows; *cap = s->cap_rows; break;
    default: return fail(PGS_ERR_INVALID_ARG, "buffer id %d", which);
  }
  return PGS_OK;
}

size_t pgs_sort_scratch_bytes(int64_t n_max) { return sort_scratch_layout(nullptr, n_max, 9).bytes; }

pgs_status pgs_sort_pairs(uint32_t* d_keys, uint32_t* d_vals, uint32_t* d_keys_alt, uint32_t* d_vals_alt,
                          const int64_t* d_n, int64_t n_max, int bit_lo, int bit_hi, void* d_scratch,
                          size_t scratch_bytes, uint32_t* d_err, cudaStream_t stream) {
  if (!d_keys || !d_vals || !d_keys_alt || !d_vals_alt || !d_n || !d_scratch)
    return fail(PGS_ERR_INVALID_ARG, "null pointer");
  if (n_max < 0 || n_max >= (1ll << 30)) return fail(PGS_ERR_INVALID_ARG, "n_max must be in [0, 2^30)");
  if (bit_lo < 0 || bit_hi > 32 || bit_lo >= bit_hi)
    return fail(PGS_ERR_INVALID_ARG, "bit range [%d, %d)", bit_lo, bit_hi);
  SortScratch ss = sort_scratch_layout(d_scratch, n_max, 9);
  if (scratch_bytes < ss.bytes) return fail(PGS_ERR_INVALID_ARG, "scratch %zu < %zu bytes", scratch_bytes, ss.bytes);
  const int ns = device_sm_count();
  PGS_CUDA(launch_sort_pairs(d_keys, d_vals, d_keys_alt, d_vals_alt, reinterpret_cast<const long long*>(d_n), n_max,
                             bit_lo, bit_hi, ss, d_err ? d_err : ss.err, kDefaultSpinLimit, kNoHoldTile, ns, stream));
  return PGS_OK;
}

size_t pgs_scan_scratch_bytes(void) { return kScanBlocks * sizeof(unsigned long long); }

pgs_status pgs_exclusive_scan_u32(const uint32_t* d_in, const uint32_t* d_index, uint32_t* d_out,
                                  unsigned long long* d_total, const int64_t* d_n, void* d_scratch,
                                  size_t scratch_bytes, cudaStream_t stream) {
  if (!d_in || !d_out || !d_total || !d_n || !d_scratch) return fail(PGS_ERR_INVALID_ARG, "null pointer");
  if (scratch_bytes < pgs_scan_scratch_bytes()) return fail(PGS_ERR_INVALID_ARG, "scratch too small");
  launch_exclusive_scan(d_in, d_index, d_out, d_total, reinterpret_cast<const long long*>(d_n),
                        static_cast<unsigned long long*>(d_scratch), stream);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

}  // extern "C"
