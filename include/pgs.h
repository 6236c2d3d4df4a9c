/*
 * pgs.h -- C ABI of the single-GPU (sm_103a) hot path of the batch-level
 * RGB-Depth-Normal training step over the hybrid anchor / voxel Gaussian
 * representation (PH^2-3D) of CityGS-X.
 *
 * The step is: LoD + frustum cull of anchors (Sec. 3.1, Octree-GS paragraph)
 * -> shared decoder F_de turning each visible anchor into n = 10 Gaussians
 * (Eq. 4) -> EWA projection -> tile binning and a radix sort by (tile, depth)
 * (the reorder pi of Eq. 5) -> front-to-back blending of RGB (Eq. 5), normal
 * (Eq. 6) and distance / unbiased depth (Eq. 7) -> batch losses (Eq. 8-9 plus
 * a normal-depth consistency term) -> reverse-order backward to the anchor
 * and decoder parameters.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every pointer named d_* or held in a *_ptrs struct is a DEVICE pointer
 *    owned by the caller; the library never frees it.  The library owns only
 *    its workspace, allocated in pgs_scene_create and freed in
 *    pgs_scene_destroy.  Host pointers (descriptors, camera arrays) are read
 *    during the call only.
 *  - Cameras: OpenCV frame (x right, y down, z forward); R maps world to
 *    camera (row-major 3x3), x_cam = R x_world + t; pixel centres sit at
 *    (u + 0.5, v + 0.5).
 *  - Images of a batch live in one ragged arena: view v occupies pixels
 *    [pix_off[v], pix_off[v] + W_v H_v) with pix_off[v] = sum_{u<v} W_u H_u.
 *    Single-channel maps are [pix] (row-major H x W per view); 3-channel maps
 *    are planar per view: channel c of view v starts at 3 pix_off[v] + c W_v H_v.
 *  - Gradient outputs are ACCUMULATED into (+=); the caller zeroes them.
 *  - Calls that take a cudaStream_t only enqueue work on it: they never
 *    synchronise, allocate or read back, so a sequence of them can be captured
 *    into a CUDA graph.  Argument errors are returned at once; errors found by
 *    the GPU (capacity overflow, a bounded wait that ran out, non-finite
 *    values) raise a device flag that pgs_read_status returns.
 *  - Status codes: PGS_OK = 0, otherwise one of pgs_status_code; the message
 *    of the last failing call on this host thread is pgs_last_error().
 */
#ifndef PGS_H_
#define PGS_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pgs_status;
enum pgs_status_code {
  PGS_OK = 0,
  PGS_ERR_INVALID_ARG = 1,   /* bad pointer, size or descriptor field */
  PGS_ERR_CAPACITY = 2,      /* rows / pairs exceeded the capacities given at create */
  PGS_ERR_TIMEOUT = 3,       /* a bounded device-side wait (sort look-back) ran out */
  PGS_ERR_NONFINITE = 4,     /* non-finite value met in a parameter, a loss or a gradient */
  PGS_ERR_CUDA = 5,          /* a CUDA runtime call failed */
  PGS_ERR_UNSUPPORTED = 6,   /* valid request the library does not handle */
  PGS_ERR_BOUNDS = 7         /* an index failed a bounds check (bounds-checked build only; the access was skipped) */
};

#define PGS_MAX_VIEWS 32
#define PGS_N_OFFSETS 10
#define PGS_FEAT_DIM 32
#define PGS_HIDDEN 32
#define PGS_OUT_DIM 110

enum pgs_mode { PGS_MODE_EXPLICIT = 0, PGS_MODE_ANCHOR = 1 };
/* Arithmetic of the decoder F_de (Eq. 4; the paper does not state one).
 *  FP32:       FP32 SIMT.
 *  BF16:       the 5th-generation tensor cores, BF16 operands and FP32
 *              accumulation.  The colour heads take one BF16 pass (their error
 *              reaches the image through a sigmoid and stays below 1e-3);
 *              layer 1 and the opacity, scale and rotation heads, which decide
 *              the blend weights, the smallest-scale normal axis of Eq. 6 and
 *              the normalised rotation, use an exact three-piece BF16 split of
 *              both operands (six products per layer: FP32-accurate).
 *  BF16_1PASS: every product in one BF16 pass (a precision study: its normal
 *              and depth maps move by up to ~1e-1, far past the colour bar). */
enum pgs_decode_precision { PGS_DECODE_FP32 = 0, PGS_DECODE_BF16 = 1, PGS_DECODE_BF16_1PASS = 2 };

typedef struct pgs_camera {
  float R[9];        /* world -> camera rotation, row-major */
  float t[3];        /* translation, x_cam = R x_world + t */
  float fx, fy, cx, cy;
  int32_t width, height;
} pgs_camera;

/* Thresholds of the blending rules (3DGS, which Sec. 3.1 builds on) and of
 * the LoD rule (Sec. 3.1).  pgs_default_params fills the values the library
 * is tested with: near 0.01, dilation 0.3 px^2, alpha in [1/255, 0.99], stop
 * before T drops below 1e-4, J clamp 1.3 tan(fov/2), tile-list pad 1e-3, bg 0. */
typedef struct pgs_render_params {
  float near_plane;
  float dilation;
  float alpha_min;
  float alpha_max;
  float t_min;
  float jclamp;
  float tile_pad;      /* the tile list of a Gaussian is its ln(255 o) + tile_pad level set */
  float lod_d0;        /* anchor at level k active iff k <= clamp(floor(log2(d0/d)), 0, K-1) */
  int32_t n_levels;    /* K */
  float bg;            /* background value of the RGB channels (depth / normal have none) */
  int32_t tile_w;      /* 16 x 16 default; 8 x 32 and 32 x 8 also accepted */
  int32_t tile_h;
  int32_t decode_precision;   /* pgs_decode_precision (anchor mode) */
  int32_t in_dim;      /* decoder input: 35 = feature + unit view direction (36 adds distance) */
  int32_t blend_batch; /* Gaussians staged in shared memory per round of the forward blend:
                          128, 256 (default) or 512; no effect on the results */
} pgs_render_params;

typedef struct pgs_scene_desc {
  int32_t mode;                 /* pgs_mode */
  int64_t n_primitives;         /* explicit: Gaussians; anchor: anchors (< 2^27) */
  int32_t max_views;            /* <= PGS_MAX_VIEWS */
  int64_t max_pixels;           /* sum of W_v H_v over a batch */
  int64_t capacity_rows;        /* anchor mode: visible (view, anchor) rows */
  int64_t capacity_pairs;       /* (Gaussian-view, tile) pairs, < 2^30 */
  pgs_render_params params;
} pgs_scene_desc;

typedef struct pgs_explicit_ptrs {   /* N Gaussians, float32, caller-owned */
  const float* means;           /* [N,3] world */
  const float* log_scales;      /* [N,3] */
  const float* quats;           /* [N,4] (w,x,y,z), normalised on use */
  const float* opacity_logits;  /* [N]  opacity = sigmoid(.) */
  const float* colors;          /* [N,3] used as given */
} pgs_explicit_ptrs;

typedef struct pgs_anchor_ptrs {     /* N anchors (Sec. 3.2), caller-owned */
  const float* x;               /* [N,3] voxel position x_v */
  const int32_t* level;         /* [N]   LoD level k */
  const float* log_l;           /* [N,3] log of the scaling factor l_v */
  const float* offsets;         /* [N,10,3] learnable offsets O_v */
  const float* feat;            /* [N,32] embedding F_v, 16-byte aligned */
} pgs_anchor_ptrs;

typedef struct pgs_mlp_ptrs {        /* shared decoder F_de (Eq. 4): 35 -> 32 (ReLU) -> 110 */
  const float* W1;              /* [32, in_dim] row-major (out x in) */
  const float* b1;              /* [32] */
  const float* W2;              /* [110, 32] */
  const float* b2;              /* [110] */
} pgs_mlp_ptrs;

typedef struct pgs_image_ptrs {      /* per-pixel outputs of pgs_render_batch (arena layout) */
  float* rgb;                   /* [3 x pix] Eq. 5 */
  float* depth;                 /* [pix] unbiased depth D_hat, Eq. 7 (0 where guarded) */
  float* normal;                /* [3 x pix] un-normalised N_hat, Eq. 6, camera frame */
  float* dist;                  /* [pix] blended plane distance D, Eq. 7 */
  float* t_final;               /* [pix] final transmittance */
  uint32_t* last;               /* [pix] 1 + sorted-list index of the last contributor (0: none) */
  uint32_t* n_contrib;          /* [pix] number of contributing Gaussians (may be NULL) */
  uint32_t* n_eval;             /* [pix] pairs evaluated before the pixel stopped (may be NULL) */
} pgs_image_ptrs;

typedef struct pgs_image_grad_ptrs { /* dL/d outputs (arena layout) */
  float* rgb;                   /* [3 x pix] */
  float* depth;                 /* [pix] w.r.t. D_hat */
  float* normal;                /* [3 x pix] w.r.t. N_hat */
} pgs_image_grad_ptrs;

typedef struct pgs_target_ptrs {
  const float* rgb;             /* [3 x pix] target colour */
  const float* prior;           /* [pix] depth prior */
  const float* mask;            /* [pix] 1 where the prior is trusted, else 0 */
} pgs_target_ptrs;

typedef struct pgs_loss_params {
  float lambda_depth;           /* 1.0 */
  float lambda_normal;          /* 0.1 */
} pgs_loss_params;

typedef struct pgs_param_grad_ptrs { /* accumulated (+=); NULL entries are skipped */
  /* explicit mode */
  float* means; float* log_scales; float* quats; float* opacity_logits; float* colors;
  /* anchor mode */
  float* x; float* log_l; float* offsets; float* feat;
  float* W1; float* b1; float* W2; float* b2;
} pgs_param_grad_ptrs;

typedef struct pgs_stats {           /* counts of the last pgs_render_batch */
  int64_t rows;                 /* visible (view, anchor) rows (anchor mode) */
  int64_t gaussian_views;       /* Gaussian-view slots projected */
  int64_t launches;             /* kernels this scene has enqueued since create (memsets excluded) */
  int64_t pairs;                /* (Gaussian-view, tile) pairs P */
  int64_t tiles;                /* tiles of the batch */
  int64_t pixels;
  uint32_t flags;               /* device error flags (bit i = status code i) */
} pgs_stats;

typedef struct pgs_scene pgs_scene;

const char* pgs_last_error(void);
const char* pgs_status_string(pgs_status s);
/* 1 in the bounds-checked build of the library (libpgs_checked.so, compiled
 * with PGS_CHECKED: the blend, sort, emission and range kernels check their
 * list, range, record and pixel indices against the scene's allocations and
 * raise PGS_ERR_BOUNDS instead of accessing out of range), 0 otherwise. */
int pgs_checked_build(void);
void pgs_default_params(pgs_render_params* p);

/* Validate the descriptor, allocate the workspace sized by its capacities.
 * Errors: PGS_ERR_INVALID_ARG (out of range field), PGS_ERR_CUDA (allocation). */
pgs_status pgs_scene_create(const pgs_scene_desc* desc, pgs_scene** out);
void pgs_scene_destroy(pgs_scene* s);

/* Bind caller-owned parameter buffers (device pointers kept until rebound):
 * explicit 3D Gaussians, or the anchors of Sec. 3.2 and the decoder F_de. */
pgs_status pgs_scene_bind_explicit(pgs_scene* s, const pgs_explicit_ptrs* p);
pgs_status pgs_scene_bind_anchors(pgs_scene* s, const pgs_anchor_ptrs* a, const pgs_mlp_ptrs* w);

/* Decoder only (Eq. 4): for each view, every LoD-active anchor whose bound
 * meets the frustum is decoded into 10 Gaussians.  Writes row r = (view,
 * anchor) packed as view << 27 | anchor into d_rows[r] and, for Gaussian
 * j of row r (index 10 r + j): d_mu [.,3], d_opacity [.], d_color [.,3],
 * d_scale [.,3], d_quat [.,4] (unit).  *d_n_rows (device int64) receives the
 * row count; rows beyond capacity_rows are dropped and flag PGS_ERR_CAPACITY.
 * Output buffers hold capacity_rows rows (x 10 Gaussians). */
pgs_status pgs_decode_anchors(pgs_scene* s, const pgs_camera* cams, int n_views, uint32_t* d_rows,
                              float* d_mu, float* d_opacity, float* d_color, float* d_scale, float* d_quat,
                              int64_t* d_n_rows, cudaStream_t stream);

/* Forward of the whole batch: cull + decode + project, bin and sort by
 * (view tile, FP32 depth, index), blend (Eq. 5-7).  The sorted lists and
 * per-Gaussian records stay in the workspace for pgs_backward.
 * rgb, depth, normal, dist, t_final and last are required. */
pgs_status pgs_render_batch(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* out,
                            cudaStream_t stream);

/* Loss of the rendered batch and dL/d(rgb, depth, normal) (Eq. 8-9 and the
 * consistency term; 1/B batch mean).  d_loss[4] receives (total, rgb,
 * depth, normal); the image gradients are OVERWRITTEN (not accumulated). */
pgs_status pgs_loss_grad(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* img,
                         const pgs_target_ptrs* tgt, const pgs_loss_params* lp, float* d_loss,
                         const pgs_image_grad_ptrs* grad, cudaStream_t stream);

/* Reverse-order backward of the last pgs_render_batch (Eq. 5-7 walked back
 * to front, then the projection and Eq. 4): transmittance is recomputed from
 * t_final and last (no per-pair state is stored).  The cameras must equal
 * those of that render.  Parameter gradients are accumulated. */
pgs_status pgs_backward(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* img,
                        const pgs_image_grad_ptrs* grad, const pgs_param_grad_ptrs* pg, cudaStream_t stream);

/* Synchronise the stream, return the first device-raised error and clear it. */
pgs_status pgs_read_status(pgs_scene* s, cudaStream_t stream);
/* Synchronise the stream and report the counts of the last render. */
pgs_status pgs_get_stats(pgs_scene* s, pgs_stats* out, cudaStream_t stream);

/* Per-stage timing (profiling aid, no counterpart in the paper).  With
 * profiling on, every stage of the following calls is bracketed by CUDA
 * events on the launching stream (recorded as external event nodes when the
 * stream is being captured into a graph).  pgs_get_stage_times waits for
 * those events and writes the most recent duration of each stage in ms (-1
 * if it did not run) for the first n of PGS_N_STAGES stages.  Profiling also
 * opens an NVTX range named after the stage ("pgs:blend_bwd", ...) around the
 * host-side enqueue of each stage, for timeline tools; with no NVTX tool
 * attached those calls do nothing. */
enum pgs_stage {
  PGS_STAGE_PROJECT = 0,      /* cull + decode + projection + tile counts */
  PGS_STAGE_DEPTH_SORT = 1,   /* radix sort of the Gaussian-views by depth */
  PGS_STAGE_BIN = 2,          /* offsets scan + (tile, Gaussian) pair emission */
  PGS_STAGE_TILE_SORT = 3,    /* stable radix sort of the pairs by tile + tile ranges */
  PGS_STAGE_BLEND_FWD = 4,
  PGS_STAGE_LOSS = 5,
  PGS_STAGE_BLEND_BWD = 6,
  PGS_STAGE_PROJECT_BWD = 7,  /* projection (+ decoder input/activation) backward */
  PGS_STAGE_WGRAD = 8,        /* decoder weight-gradient reduction */
  PGS_STAGE_PRIOR = 9,        /* enhanced depth prior (pgs_filter_depth_prior) */
  PGS_STAGE_NCC = 10,         /* batch geometric NCC loss (pgs_ncc_loss_grad) */
  PGS_STAGE_TSDF = 11,        /* TSDF fusion (pgs_tsdf_integrate) */
  PGS_N_STAGES = 12
};
pgs_status pgs_set_profiling(pgs_scene* s, int enable);

/* Bounded device waits (no counterpart in the paper).  The only spin-waits of
 * the step are the look-backs of the onesweep sorts (depth, tile and queue
 * order): each gives up after spin_limit polls (0 restores the default,
 * 2^20), raises PGS_ERR_TIMEOUT for pgs_read_status and leaves that sort's
 * output unspecified; the step then continues on safe stand-ins (Gaussians in
 * index order, no pairs, tiles in index order), so every later call of the
 * step returns and the context stays usable, but the images and gradients of
 * that step are meaningless.  withhold_tile is a failure-path test hook: the
 * onesweep tile (4096 keys) with this index never publishes its look-back
 * status in any pass, so the next tile's wait runs out; PGS_NO_WITHHELD_TILE
 * (the default) publishes every tile.  Applies to later calls on this scene. */
#define PGS_NO_WITHHELD_TILE 0xffffffffu
pgs_status pgs_scene_set_wait_limits(pgs_scene* s, uint32_t spin_limit, uint32_t withhold_tile);
pgs_status pgs_get_stage_times(pgs_scene* s, float* ms, int n);

/* Launch-shape autotuner (no counterpart in the paper: it only picks how the
 * work of Eq. 5-7 is laid out on the GPU, never what is computed).  For every
 * tile shape (16x16, 8x32, 32x8) and forward shared-memory batch (128, 256,
 * 512 Gaussians) it runs pgs_render_batch + pgs_backward on the caller's
 * batch and buffers once untimed and `reps` times timed with CUDA events on
 * `stream`, keeps the combination with the smallest median time in the
 * scene's parameters, and caches it per workload signature (device, mode,
 * number of primitives, view resolutions): a later call with the same
 * signature applies the cached choice without timing.  Images and buffers
 * are laid out as for pgs_render_batch / pgs_backward; afterwards the images
 * hold the last render and the parameter gradients hold the sum of all the
 * tuning passes (zero them before the next step).  If `entries` is not null
 * it receives up to max_entries timed combinations (ms < 0 when the choice
 * came from the cache) and *n_entries their number.  Synchronises the
 * stream; PGS_ERR_INVALID_ARG while the stream is being captured. */
typedef struct pgs_tune_entry {
  int32_t tile_w, tile_h, blend_batch;
  float ms;                     /* median of the timed render + backward passes */
} pgs_tune_entry;
pgs_status pgs_autotune(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* img,
                        const pgs_image_grad_ptrs* grad, const pgs_param_grad_ptrs* pg, int reps,
                        pgs_tune_entry* entries, int max_entries, int* n_entries, cudaStream_t stream);
/* Enhanced depth prior (Step 2 of the batch-level progressive training,
 * Sec. 3.4; the threshold tau_d = 1 is given in the supplementary
 * implementation details).  For the batch `cams`:
 *  1. per view, the scale and shift of the pseudo depth D_p that fit the
 *     sparse points' view depths by least squares (points sampled bilinearly
 *     in D_p where they project): D~_p = s D_p + t;
 *  2. per pixel, the re-projection error E: the pixel's 3D point at depth D~_p
 *     is projected into each of the view's k nearest batch views (by camera
 *     centre), lifted there with that view's D~_p (bilinear), projected back;
 *     E = the smallest pixel distance over the neighbours where the round trip
 *     is defined;
 *  3. D~_f = D~_p where E <= tau_d or no neighbour could check the pixel, else
 *     0 (also 0 where D_p <= 0); mask = 1 where D~_f is kept.
 * d_pseudo: per-pixel pseudo depth in the image arena layout (<= 0 = none);
 * d_points: float[n_points][3] world points (the sparse cloud); outputs, all
 * device and caller-owned: d_prior_out and d_mask_out [pixels] (the loss's
 * depth prior and mask), d_scale_shift float[n_views][2] ((1, 0) for a view
 * with fewer than two usable points), d_err_out [pixels] optional (E, or -1
 * where unchecked).  k_neighbors in 1..4 (clamped to n_views - 1), tau_d > 0
 * in pixels.  Uses the scene's render parameters (near plane) and a
 * workspace area of its own: it reads nothing that pgs_render_batch writes,
 * so it may run on another stream concurrently with the render (the loss
 * that reads its outputs must then wait for it); any other two calls on one
 * scene must be ordered. */
typedef struct pgs_prior_params {
  float tau_d;
  int32_t k_neighbors;
} pgs_prior_params;
pgs_status pgs_filter_depth_prior(pgs_scene* s, const pgs_camera* cams, int n_views, const float* d_pseudo,
                                  const float* d_points, int64_t n_points, const pgs_prior_params* pp,
                                  float* d_prior_out, float* d_mask_out, float* d_scale_shift, float* d_err_out,
                                  cudaStream_t stream);

/* Batch geometric NCC loss (Step 3 of the batch-level progressive training,
 * Sec. 3.4, Eq. 10) of a rendered batch, with its gradients.
 *  - pairs: views (2i+1, 2i) for i < n_views / 2; view 2i+1 is the reference
 *    whose patches are compared, view 2i the partner (an odd last view is
 *    unpaired);
 *  - d_centers: uint32 [n_views / 2][n_per_pair] patch centres drawn by the
 *    caller (the random draw of Eq. 10), as local pixel indices y W + x of the
 *    pair's reference view;
 *  - each patch is the 7 x 7 block of reference pixels around its centre,
 *    mapped into the partner by the homography of the plane through the
 *    centre's back-projection (rendered D_hat) with the rendered normal N_hat
 *    there; NCC = S_ab / sqrt((S_aa + eps)(S_bb + eps)) over the centred sums
 *    of the BT.601 luma of the reference pixels (a) and of the partner read
 *    bilinearly at the warped positions (b, pixel centres at +1/2);
 *  - a patch is used when it lies inside the reference frame, D_hat > 0 and
 *    |N_hat . K^-1 p~| >= 1e-8 at its centre, and every warped sample has the
 *    plane in front of both cameras and its bilinear footprint inside the
 *    partner frame; centres outside the reference view give unused patches;
 *  - L_ncc = (1 / (n_views / 2)) sum over pairs of the mean of (1 - NCC) over
 *    the pair's used patches (a pair without any adds 0).
 * The partner's colours are under stop-gradient.  geometric = 1: the warped
 * positions stay differentiable, so the gradient also reaches D_hat and N_hat
 * at each patch centre; geometric = 0: the whole sampled partner patch is a
 * constant and only the reference colours receive gradients.
 * img: rgb, depth (D_hat) and normal (N_hat) of the rendered batch (other
 * fields unused).  Outputs (device, caller-owned): d_ncc float[n_views / 2]
 * [n_per_pair] the NCC of each patch, or -2 for an unused one (required: the
 * kernels keep the validity of each patch there); d_loss float[2] =
 * (lambda_ncc * L_ncc, L_ncc); gradients ACCUMULATED (+=) into grad->rgb of
 * the reference views and, in the geometric form, grad->depth and
 * grad->normal at the patch centres, scaled by lambda_ncc.  Call it after
 * pgs_loss_grad (which overwrites the gradients) and before pgs_backward.
 * Errors: PGS_ERR_INVALID_ARG for null pointers, n_per_pair outside
 * 0..2^26, eps < 0. */
typedef struct pgs_ncc_params {
  float lambda_ncc;             /* weight of L_ncc in the total loss (0.2 at the end of the paper's schedule) */
  float eps;                    /* added to each centred sum of squares (1e-6) */
  int32_t geometric;            /* 1: gradients reach D_hat and N_hat through the warp; 0: colours only */
} pgs_ncc_params;
pgs_status pgs_ncc_loss_grad(pgs_scene* s, const pgs_camera* cams, int n_views, const pgs_image_ptrs* img,
                             const uint32_t* d_centers, int64_t n_per_pair, const pgs_ncc_params* np,
                             float* d_ncc, float* d_loss, const pgs_image_grad_ptrs* grad, cudaStream_t stream);

/* Projective TSDF fusion of rendered depth and colour into a voxel volume
 * (supplementary, mesh reconstruction: voxel 0.01, truncation 0.04 for the
 * aerial scenes; the paper cites Zeng et al.'s TSDF fusion).  For each voxel
 * (i, j, k), centred at origin + (i + 1/2, j + 1/2, k + 1/2) * voxel, and each
 * view in batch order: camera depth z of the centre > near plane (the scene's
 * render parameters); its nearest pixel (floor of the projection, pixel
 * centres at +1/2) inside the frame with depth D > 0; sdf = D - z >= -trunc;
 * then tsdf <- (tsdf W + min(1, sdf / trunc)) / (W + 1), colour likewise with
 * the pixel's colour, W <- W + 1.  Voxels no view updates are not written.
 * d_depth: per-pixel z-depth in the image arena layout (D_hat of a render,
 * <= 0 = none); d_rgb: [3 x pix] colour (may be NULL, then d_color must be
 * NULL too).  Volume state (device, caller-owned, x fastest: linear index
 * (k ny + j) nx + i): d_tsdf and d_weight float[n], d_color float[n][3] or
 * NULL; initialise weight to 0 and tsdf / colour to finite values (0) before
 * the first call; later calls keep fusing.  With colour, and when the scene's
 * pair capacity holds 4 x the batch's pixels, the call first interleaves depth
 * and colour into the scene's tile-sort scratch (free between renders), so
 * like every call on a scene it must not overlap another call on the same
 * scene.  Errors: PGS_ERR_INVALID_ARG for null pointers, dims < 1 or more than
 * 2^34 voxels, voxel <= 0 or trunc <= 0. */
typedef struct pgs_tsdf_volume {
  float origin[3];              /* world position of the corner of voxel (0, 0, 0) */
  float voxel;                  /* voxel edge length */
  int32_t dims[3];              /* nx, ny, nz */
  float trunc;                  /* truncation band of the signed distance */
} pgs_tsdf_volume;
pgs_status pgs_tsdf_integrate(pgs_scene* s, const pgs_camera* cams, int n_views, const float* d_depth,
                              const float* d_rgb, const pgs_tsdf_volume* vol, float* d_tsdf, float* d_weight,
                              float* d_color, cudaStream_t stream);

/* The scene's current render parameters (as created, or as the autotuner set them). */
pgs_status pgs_scene_get_params(const pgs_scene* s, pgs_render_params* out);

/* Workspace buffers of the last render, for tests and tools (device
 * pointers owned by the scene, valid until the next render or destroy):
 * which = 0 records float[G][16], 1 tile counts uint32[G], 2 sorted pair
 * tiles uint32[P], 3 sorted pair Gaussian ids uint32[P], 4 tile ranges
 * uint32[T][2], 5 depth-sorted Gaussian ids uint32[G], 6 rows uint32[rows]. */
pgs_status pgs_scene_buffer(pgs_scene* s, int which, void** d_ptr, int64_t* capacity_elems);

/* Stand-alone stages of the reorder pi (Eq. 5), exposed for the integer
 * parity tests and for reuse.
 *
 * Stable LSD radix sort (one histogram pass, then one pass per 8-bit digit,
 * or two 9-bit digits for ranges of 17-18 bits, one pass fewer;
 * decoupled look-back) of n = *d_n (device int64, clamped to n_max)
 * key/value pairs on bits [bit_lo, bit_hi) of the keys.  The sorted result
 * ends in (d_keys, d_vals); d_keys_alt / d_vals_alt are ping-pong buffers of
 * the same size.  Scratch must hold pgs_sort_scratch_bytes(n_max) bytes.  A
 * look-back wait that runs out (never expected) ORs bit PGS_ERR_TIMEOUT (the
 * value 1u << PGS_ERR_TIMEOUT) into *d_err (device uint32, may be NULL) and
 * the pass completes with an unspecified order.  *d_err must be 0 on entry:
 * the passes poll it and stop waiting once that bit is set. */
size_t pgs_sort_scratch_bytes(int64_t n_max);
pgs_status pgs_sort_pairs(uint32_t* d_keys, uint32_t* d_vals, uint32_t* d_keys_alt, uint32_t* d_vals_alt,
                          const int64_t* d_n, int64_t n_max, int bit_lo, int bit_hi, void* d_scratch,
                          size_t scratch_bytes, uint32_t* d_err, cudaStream_t stream);

/* Exclusive prefix sum of n = *d_n (device) uint32 values (optionally
 * gathered: value k = d_in[d_index[k]]); *d_total (device uint64) = sum.
 * Scratch must hold pgs_scan_scratch_bytes() bytes. */
size_t pgs_scan_scratch_bytes(void);
pgs_status pgs_exclusive_scan_u32(const uint32_t* d_in, const uint32_t* d_index, uint32_t* d_out,
                                  unsigned long long* d_total, const int64_t* d_n, void* d_scratch,
                                  size_t scratch_bytes, cudaStream_t stream);

/* The same radix sort for callers that cannot allocate device memory (no
 * counterpart in the paper): code running inside an allocator or memory-pool
 * callback, plug-ins whose host framework owns all device memory, real-time
 * paths that must not risk an allocation failure.  Sorts n (host value,
 * 0 <= n <= 1048576) key/value pairs in place on bits [bit_lo, bit_hi), with
 * the same stable order as pgs_sort_pairs.  All scratch (histograms,
 * look-back status, ping-pong keys and values) sits in one fixed array of
 * about 9.4 MB inside the library's device image, which every GPU that loads
 * the library holds until the process exits; the call allocates and frees
 * nothing.  Each call looks up that array's device address on the current
 * device.  Warm-up: under CUDA's lazy module loading the FIRST call on a
 * device may load the library's device code (which is when the array is
 * reserved) and sets up the sort's launch once, so the allocation-free
 * guarantee holds from the second call on; make one warm-up call (any
 * n >= 1) per device first, and make it outside any stream capture.  Every
 * call on a device shares the array and it keeps the last call's contents,
 * so calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them.  n = 0 does nothing (keys and values may then be NULL).
 * Larger n is rejected with PGS_ERR_INVALID_ARG and a message in
 * pgs_last_error().  A look-back wait that runs out ORs bit PGS_ERR_TIMEOUT
 * (the value 1u << PGS_ERR_TIMEOUT) into *d_err (device uint32, may be NULL,
 * then an internal word is used).  A caller-supplied *d_err must be 0 on
 * entry: the sort polls it and gives up its look-back waits early (leaving an
 * unspecified order) once that bit is set. */
pgs_status pgs_sort_pairs_noalloc(uint32_t* d_keys, uint32_t* d_vals, int64_t n, int bit_lo, int bit_hi,
                                  uint32_t* d_err, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* PGS_H_ */
