// Internal declarations shared by the CUDA translation units of libpgs.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/pgs.h"

namespace pgs {

constexpr int kMaxViews = PGS_MAX_VIEWS;
constexpr int kNOff = PGS_N_OFFSETS;
constexpr int kFeat = PGS_FEAT_DIM;
constexpr int kHidden = PGS_HIDDEN;
constexpr int kOut = PGS_OUT_DIM;
constexpr int kMaxIn = 36;

// device error flag bits (bit = status code)
constexpr uint32_t kFlagCapacity = 1u << PGS_ERR_CAPACITY;
constexpr uint32_t kFlagTimeout = 1u << PGS_ERR_TIMEOUT;
constexpr uint32_t kFlagNonfinite = 1u << PGS_ERR_NONFINITE;
constexpr uint32_t kFlagBounds = 1u << PGS_ERR_BOUNDS;

// log2(e): the blend evaluates alpha = o * 2^(log2e * power)
constexpr float kLog2e = 1.4426950408889634f;

struct ViewDev {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float center[3];     // camera centre in world
  float lim_x, lim_y;  // J clamp on x/z and y/z
  int W, H;
  int tiles_x, tiles_y;
  int tile_base;       // first global tile id of this view
  long long pix_off;   // first pixel of this view in the arena
};

struct ParamsDev {
  float near_plane, dilation, alpha_min, alpha_max, t_min, jclamp, tile_pad, lod_d0, bg;
  int n_levels, tile_w, tile_h, in_dim, blend_batch;
  int decode;          // pgs_decode_precision of the decoder forward (the backward follows its rounding)
};

struct BatchDev {
  ViewDev v[kMaxViews];
  ParamsDev p;
  int n_views;
  int total_tiles;
  long long total_pixels;
  long long cap_pairs, cap_g;   // allocated pair and Gaussian-view slots of the scene (bounds of the checked build)
  uint32_t* flags;              // the scene's device error flags
};

// Gaussian-view record: 4 x float4 = 64 B
//  r0 = (mx_hi, my_hi, mx_lo, my_lo)   2D mean relative to (cx, cy), double-float
//  r1 = (A, B, C, opacity)             conic (inverse 2D covariance), natural units
//  r2 = (r, g, b, d)                   colour, plane distance d = n . mu_c
//  r3 = (nx, ny, nz, z)                camera-frame normal facing the camera, view depth
constexpr int kRecF4 = 4;

// grad record: 4 x float4 = 64 B
//  (dmx, dmy, dA, dB), (dC, dopacity, dr, dg), (db, dd, dnx, dny), (dnz, 0, 0, 0)
constexpr int kGradFields = 13;

__device__ __forceinline__ int view_of_tile(const BatchDev& b, int tile) {
  int v = 0;
#pragma unroll 1
  for (int i = 1; i < b.n_views; ++i)
    if (tile >= b.v[i].tile_base) v = i;
  return v;
}

__device__ __forceinline__ int view_of_pixel(const BatchDev& b, long long p) {
  int v = 0;
#pragma unroll 1
  for (int i = 1; i < b.n_views; ++i)
    if (p >= b.v[i].pix_off) v = i;
  return v;
}

// 1/x with the hardware approximation (about 1 ulp), denormals flushed
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void set_flag(uint32_t* flags, uint32_t bit) { atomicOr(flags, bit); }

// Index checks of the bounds-checked build (compiled with -DPGS_CHECKED, library libpgs_checked.so): a
// failing check raises PGS_ERR_BOUNDS in *flags and returns false, and the caller skips the access.  In the
// production build every check is the constant true and costs nothing.
#ifdef PGS_CHECKED
constexpr bool kChecked = true;
__device__ __forceinline__ bool in_bounds(bool ok, uint32_t* flags) {
  if (!ok && flags) set_flag(flags, kFlagBounds);
  return ok;
}
#else
constexpr bool kChecked = false;
__device__ __forceinline__ constexpr bool in_bounds(bool, uint32_t*) { return true; }
#endif

// ---- packed FP32 pairs (sm_100 family): add / sub / mul / fma .rn.f32x2 round each half exactly as the
// scalar __fadd_rn / __fsub_rn / __fmul_rn / __fmaf_rn would, at one issue slot for both halves
struct f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 f2_make(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ f2 f2_splat(float x) { return f2_make(x, x); }
__device__ __forceinline__ float f2_lo(f2 a) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
  return lo;
}
__device__ __forceinline__ float f2_hi(f2 a) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
  return hi;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ f2 f2_shfl_xor(f2 a, int m) {
  return f2_make(__shfl_xor_sync(0xffffffffu, f2_lo(a), m), __shfl_xor_sync(0xffffffffu, f2_hi(a), m));
}

// ---- error-free transforms (Knuth TwoSum, FMA TwoProduct) for the 2D mean
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// compensated dot product a . b + c + extra (Ogita, Rump, Oishi "Dot2") -> (hi, lo);
// "extra" carries small terms (a . b_lo of a double-float b) into the error sum
__device__ __forceinline__ void dot3_add(const float* a, float b0, float b1, float b2, float c, float& hi,
                                         float& lo, float extra = 0.f) {
  float p = __fmul_rn(a[0], b0);
  float err = __fmaf_rn(a[0], b0, -p);
  float bs[2] = {b1, b2};
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    float h = __fmul_rn(a[i + 1], bs[i]);
    float r = __fmaf_rn(a[i + 1], bs[i], -h);
    float s, q;
    two_sum(p, h, s, q);
    p = s;
    err = __fadd_rn(err, __fadd_rn(q, r));
  }
  float s, q;
  two_sum(p, c, s, q);
  err = __fadd_rn(err, __fadd_rn(q, extra));
  fast_two_sum(s, err, hi, lo);
}
// f * (xh + xl) / (zh + zl) as a double-float
__device__ __forceinline__ void df_scaled_ratio(float f, float xh, float xl, float zh, float zl, float& mh,
                                                float& ml) {
  float qh = __fdiv_rn(xh, zh);
  float r = __fmaf_rn(-qh, zh, xh);
  r = __fadd_rn(r, __fsub_rn(xl, __fmul_rn(qh, zl)));
  float ql = __fdiv_rn(r, zh);
  float ph = __fmul_rn(f, qh);
  float pl = __fmaf_rn(f, qh, -ph);
  pl = __fmaf_rn(f, ql, pl);
  fast_two_sum(ph, pl, mh, ml);
}

// Quaternion (w,x,y,z), unit -> rotation matrix (columns are local axes in world)
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float* R) {
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// ---- tile set of a Gaussian: the tiles whose pixel-centre rectangle meets the
// ellipse 1/2 d^T Q d <= ln(255 o) + pad.  Evaluated with explicitly rounded
// operations so that the counting and the emitting kernels agree bit for bit.
struct TileEllipse {
  float mxh, mxl, myh, myl;   // mean relative to principal point (double-float)
  float A, B, C;              // conic
  float two_lvl;              // 2 (ln(255 o) + pad)
  float rx, ry;               // half extents of the ellipse
  float det;
};

__device__ __forceinline__ bool tile_ellipse_setup(const float4 r0, const float4 r1, const ParamsDev& p,
                                                   TileEllipse& e) {
  float o = r1.w;
  if (!(o >= p.alpha_min)) return false;
  float lvl = __fadd_rn(logf(__fmul_rn(255.f, o)), p.tile_pad);
  if (!(lvl > 0.f)) return false;
  e.mxh = r0.x; e.myh = r0.y; e.mxl = r0.z; e.myl = r0.w;
  e.A = r1.x; e.B = r1.y; e.C = r1.z;
  e.det = __fsub_rn(__fmul_rn(e.A, e.C), __fmul_rn(e.B, e.B));
  if (!(e.det > 0.f) || !(e.A > 0.f)) return false;
  e.two_lvl = __fmul_rn(2.f, lvl);
  // cov_xx = C / det, cov_yy = A / det
  e.rx = __fsqrt_rn(__fdiv_rn(__fmul_rn(e.two_lvl, e.C), e.det));
  e.ry = __fsqrt_rn(__fdiv_rn(__fmul_rn(e.two_lvl, e.A), e.det));
  return isfinite(e.rx) && isfinite(e.ry);
}

__device__ __forceinline__ float clamp_tile(float t) { return fminf(fmaxf(t, -1.0e6f), 1.0e6f); }

// x extent of the ellipse at offset dy from the mean: (-B dy -+ sqrt(2A lvl - det dy^2)) / A
__device__ __forceinline__ float ellipse_x_at(const TileEllipse& e, float dy, float sgn) {
  float disc = __fsub_rn(__fmul_rn(e.A, e.two_lvl), __fmul_rn(e.det, __fmul_rn(dy, dy)));
  disc = fmaxf(disc, 0.f);
  float s = __fsqrt_rn(disc);
  return __fdiv_rn(__fadd_rn(__fmul_rn(-e.B, dy), __fmul_rn(sgn, s)), e.A);
}

// Visit the tiles of the ellipse in one view: for each tile row, the contiguous
// column range [c0, c1] of touched tiles.  f(ty, c0, c1) is called per row.
// Tile rows of an ellipse: the row range [ty0, ty1] and the dy of its left and
// right extreme points; tile_row_span then gives one row's column range.
// for_each_tile_row walks the rows in order; the pair emission also splits the
// rows of large ellipses over a warp.  Both use the same per-row arithmetic.
struct TileRows {
  int ty0, ty1;
  float dy_left, dy_right;
};
__device__ __forceinline__ TileRows tile_rows(const TileEllipse& e, const ViewDev& v, int TW, int TH) {
  const float cy = v.cy;
  float my_abs = __fadd_rn(__fadd_rn(e.myh, e.myl), cy);
  float y_lo = __fsub_rn(my_abs, e.ry), y_hi = __fadd_rn(my_abs, e.ry);
  // float -> int conversions are clamped first (huge ellipses would saturate)
  int ty0 = max(0, (int)clamp_tile(floorf(__fdiv_rn(__fsub_rn(y_lo, 0.5f), (float)TH))) - 1);
  int ty1 = min(v.tiles_y - 1, (int)clamp_tile(floorf(__fdiv_rn(__fsub_rn(y_hi, 0.5f), (float)TH))) + 1);
  // left / right extreme points of the ellipse occur at these dy
  float dy_left = __fdiv_rn(__fmul_rn(e.B, e.rx), e.C);
  float dy_right = -dy_left;
  return TileRows{ty0, ty1, dy_left, dy_right};
}

__device__ __forceinline__ bool tile_row_span(const TileEllipse& e, const ViewDev& v, int TW, int TH,
                                              const TileRows& R, int ty, int& tx0_out, int& tx1_out) {
  const float cy = v.cy, cx = v.cx;
  const float dy_left = R.dy_left, dy_right = R.dy_right;
  int py0 = ty * TH, py1 = min(ty * TH + TH - 1, v.H - 1);
  // band in dy relative to the mean (double-float mean): (y_rel - mh) - ml
  float b0 = __fsub_rn(__fsub_rn(__fsub_rn((float)py0 + 0.5f, cy), e.myh), e.myl);
  float b1 = __fsub_rn(__fsub_rn(__fsub_rn((float)py1 + 0.5f, cy), e.myh), e.myl);
  if (b0 > e.ry || b1 < -e.ry) return false;
  float c0 = fmaxf(b0, -e.ry), c1 = fminf(b1, e.ry);
  float xmin = (dy_left >= c0 && dy_left <= c1) ? -e.rx : ellipse_x_at(e, dy_left < c0 ? c0 : c1, -1.f);
  float xmax = (dy_right >= c0 && dy_right <= c1) ? e.rx : ellipse_x_at(e, dy_right < c0 ? c0 : c1, 1.f);
  // tile column tx spans pixel centres [tx TW + 0.5, min(tx TW + TW - 1, W - 1) + 0.5]
  // (relative: subtract cx); touched iff x0 - m <= xmax and x1 - m >= xmin
  float ax_min = __fadd_rn(__fadd_rn(__fadd_rn(xmin, e.mxh), e.mxl), cx);
  float ax_max = __fadd_rn(__fadd_rn(__fadd_rn(xmax, e.mxh), e.mxl), cx);
  if (ax_min > (float)v.W - 0.5f || ax_max < 0.5f) return false;
  // candidate range widened by one column each side, then tightened exactly
  int tx0 = (int)clamp_tile(ceilf(__fdiv_rn(__fsub_rn(__fadd_rn(ax_min, 0.5f), (float)TW), (float)TW))) - 1;
  int tx1 = (int)clamp_tile(floorf(__fdiv_rn(__fsub_rn(ax_max, 0.5f), (float)TW))) + 1;
  tx0 = max(tx0, 0);
  tx1 = min(tx1, v.tiles_x - 1);
  while (tx0 <= tx1) {
    int px1 = min(tx0 * TW + TW - 1, v.W - 1);
    float x1 = __fsub_rn(__fsub_rn(__fsub_rn((float)px1 + 0.5f, cx), e.mxh), e.mxl);
    if (x1 >= xmin) break;
    ++tx0;
  }
  while (tx1 >= tx0) {
    float x0 = __fsub_rn(__fsub_rn(__fsub_rn((float)(tx1 * TW) + 0.5f, cx), e.mxh), e.mxl);
    if (x0 <= xmax) break;
    --tx1;
  }
  tx0_out = tx0;
  tx1_out = tx1;
  return tx0 <= tx1;
}

template <typename F>
__device__ __forceinline__ void for_each_tile_row(const TileEllipse& e, const ViewDev& v, int TW, int TH, F f) {
  const TileRows R = tile_rows(e, v, TW, TH);
  for (int ty = R.ty0; ty <= R.ty1; ++ty) {
    int tx0, tx1;
    if (tile_row_span(e, v, TW, TH, R, ty, tx0, tx1)) f(ty, tx0, tx1);
  }
}

}  // namespace pgs
