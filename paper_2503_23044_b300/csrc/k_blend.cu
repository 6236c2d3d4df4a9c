// Front-to-back blending of RGB (Eq. 5), normal (Eq. 6) and plane distance
// with the unbiased depth D_hat = D / (N . K^-1 p~) (Eq. 7), and its reverse-
// order backward.
//
// One CTA per (view, tile) of the batch: two pixels per thread, the tile's
// sorted Gaussian list staged in shared memory in rounds of 256 records.
// The decisions of the forward (skip power > 0, skip alpha < alpha_min, clamp
// at alpha_max, stop before T drops below t_min) are taken with explicitly
// rounded operations so that the backward recomputes bit-identical alphas and
// walks exactly the forward's contributors, from the last one down, undoing
// the transmittance by division (T_i = T_{i+1} / (1 - alpha_i)).
#include <algorithm>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

// scaled conic: power (log2 units) = A' dx^2 + C' dy^2 + B' dx dy
constexpr float kHalfLog2e = -0.5f * kLog2e;
constexpr float kNegLog2e = -kLog2e;
// Records staged in shared memory per round of the forward (NB: 128, 256 or
// 512, one to four per thread of the 128-thread CTA); picked by the autotuner.
template <int NB>
struct BlendSmem {
  float2 m[NB];    // mean relative to the block origin
  float4 q[NB];    // (A', B', C', opacity)
  float4 c[NB];    // (r, g, b, d)
  float4 n[NB];    // (nx, ny, nz, p_lo): p_lo = log2(alpha_min / opacity)
};

// The alpha >= alpha_min rule is taken on the exponent, o 2^p >= alpha_min <=>
// p >= log2(alpha_min / o), so pairs below it never reach the exponential.
struct RecF {
  float4 m, q, c, n;   // m: mean relative to the principal point (hi x, hi y, lo x, lo y); q, c, n as in BlendSmem
};
__device__ __forceinline__ RecF load_record(const float4* __restrict__ rec, uint32_t g, float a_min) {
  const float4* r = rec + (size_t)g * kRecF4;
  const float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3);
  RecF o;
  o.m = r0;
  o.q = make_float4(__fmul_rn(r1.x, kHalfLog2e), __fmul_rn(r1.y, kNegLog2e), __fmul_rn(r1.z, kHalfLog2e), r1.w);
  o.c = r2;
  o.n = make_float4(r3.x, r3.y, r3.z, log2f(__fdiv_rn(a_min, r1.w)));
  return o;
}
// Mean relative to a block origin (ox, oy), both relative to the principal
// point: one rounded expression shared by both passes, so that their pixel
// offsets dx = (px_local + 1/2) - m_t agree bit for bit.  The origin is that
// of the 32 x 32 pixel block holding the tile, so every supported tile shape
// gives a pixel the same offsets (and the same image).
constexpr int kOriginBlock = 32;
__device__ __forceinline__ int block_origin(int p0) { return p0 & ~(kOriginBlock - 1); }
__device__ __forceinline__ float2 tile_mean(const float4 m, float ox, float oy) {
  return make_float2(__fadd_rn(__fsub_rn(m.x, ox), m.z), __fadd_rn(__fsub_rn(m.y, oy), m.w));
}
template <int NB>
__device__ __forceinline__ void stage_record(BlendSmem<NB>& s, int slot, const float4* __restrict__ rec, uint32_t g,
                                             float a_min, float ox, float oy) {
  const RecF r = load_record(rec, g, a_min);
  s.m[slot] = tile_mean(r.m, ox, oy);
  s.q[slot] = r.q;
  s.c[slot] = r.c;
  s.n[slot] = r.n;
}

// power of the Gaussian at the pixel, with the exact operation order shared by both passes,
// from the products dx^2, dx dy, dy^2 (the backward reuses them for the conic sums)
__device__ __forceinline__ float eval_power_xy(const float4 q, float xx, float xy, float yy) {
  return __fmaf_rn(q.x, xx, __fmaf_rn(q.z, yy, __fmul_rn(q.y, xy)));
}
__device__ __forceinline__ float eval_power(const float4 q, float dx, float dy) {
  return eval_power_xy(q, __fmul_rn(dx, dx), __fmul_rn(dx, dy), __fmul_rn(dy, dy));
}

struct PixF {            // forward state of one pixel
  float T, cr, cg, cb, D, n0, n1, n2;
  uint32_t last, ncontrib, stop;
  bool done;
};

// Take (or not) one record at a pixel whose power test gave `take`, with every
// step predicated: alpha, the stop rule T_new < t_min (the pixel ends before
// this record) and the masked accumulation.
// STATS: also count the pixel's contributors and evaluations (diagnostic outputs).
template <bool STATS>
__device__ __forceinline__ void fwd_take(PixF& P, bool take, float power, float opac, const float4 c,
                                         const float4 nn, uint32_t j, float a_max, float t_min) {
  const float a_raw = __fmul_rn(opac, ex2_approx(power));
  const float alpha = fminf(a_max, a_raw);
  const float Tn = __fmul_rn(P.T, __fsub_rn(1.f, alpha));
  const bool stop = take && Tn < t_min;
  const bool cont = take && !stop;
  const float w = cont ? __fmul_rn(alpha, P.T) : 0.f;
  P.cr = fmaf(w, c.x, P.cr); P.cg = fmaf(w, c.y, P.cg); P.cb = fmaf(w, c.z, P.cb); P.D = fmaf(w, c.w, P.D);
  P.n0 = fmaf(w, nn.x, P.n0); P.n1 = fmaf(w, nn.y, P.n1); P.n2 = fmaf(w, nn.z, P.n2);
  P.T = cont ? Tn : P.T;
  P.last = cont ? j + 1 : P.last;
  if (STATS) {
    P.ncontrib += cont ? 1u : 0u;
    P.stop = stop ? j + 1 : P.stop;
  }
  P.done = P.done || stop;
}

__device__ __forceinline__ void fwd_write(const PixF& P, const ViewDev& v, const ParamsDev& p, int px, int py,
                                          uint32_t lo, const pgs_image_ptrs& out, long long total_pixels,
                                          uint32_t* flags) {
  if (px >= v.W || py >= v.H) return;
  const float fx_rel = (float)px + 0.5f - v.cx, fy_rel = (float)py + 0.5f - v.cy;
  const long long HW = (long long)v.W * v.H;
  const long long q = v.pix_off + (long long)py * v.W + px;
  const long long q3 = 3 * v.pix_off + (long long)py * v.W + px;
  if (!in_bounds(q < total_pixels, flags)) return;
  out.rgb[q3] = fmaf(P.T, p.bg, P.cr);
  out.rgb[q3 + HW] = fmaf(P.T, p.bg, P.cg);
  out.rgb[q3 + 2 * HW] = fmaf(P.T, p.bg, P.cb);
  out.normal[q3] = P.n0;
  out.normal[q3 + HW] = P.n1;
  out.normal[q3 + 2 * HW] = P.n2;
  // Eq. 7 with guards: |N . r| >= 1e-8 and accumulated weight >= 1e-6, else 0
  const float rx = fx_rel / v.fx, ry = fy_rel / v.fy;
  const float ndr = P.n0 * rx + P.n1 * ry + P.n2;
  const bool ok = fabsf(ndr) >= 1e-8f && (1.f - P.T) >= 1e-6f;
  out.depth[q] = ok ? P.D / ndr : 0.f;
  out.dist[q] = P.D;
  out.t_final[q] = P.T;
  out.last[q] = P.last;
  if (out.n_contrib) out.n_contrib[q] = P.ncontrib;
  if (out.n_eval) out.n_eval[q] = P.stop - lo;
}

// Each thread owns two vertically adjacent pixels of the tile, so one staged
// record and its dx serve both; each warp covers a compact 8 x 8 block of the
// tile, so its pixels tend to agree on which Gaussians they skip or take.
template <int TW>
__device__ __forceinline__ void warp_block_pixel(int tx, int ty, int TH, int& px, int& py0) {
  const int w = (int)threadIdx.x >> 5, l = (int)threadIdx.x & 31;
  constexpr int WX = TW / 8;
  px = tx * TW + (w % WX) * 8 + (l & 7);
  py0 = ty * TH + (w / WX) * 8 + 2 * (l >> 3);
}
template <int TW, int TH, int NB, bool STATS>
__device__ __forceinline__ void blend_fwd_tile(const BatchDev& b, int tile, BlendSmem<NB>& s,
                                               const float4* __restrict__ rec, const uint32_t* __restrict__ pair_g,
                                               const uint2* __restrict__ ranges, const pgs_image_ptrs& out) {
  constexpr int NT = TW * TH / 2;
  static_assert(NB % NT == 0, "whole records per thread per round");
  const int vi = view_of_tile(b, tile);
  const ViewDev& v = b.v[vi];
  const int lt = tile - v.tile_base;
  const int ty = lt / v.tiles_x, tx = lt - ty * v.tiles_x;
  int px, py0;
  warp_block_pixel<TW>(tx, ty, TH, px, py0);
  const int bx = block_origin(tx * TW), by = block_origin(ty * TH);
  const float ox = __fsub_rn((float)bx, v.cx), oy = __fsub_rn((float)by, v.cy);
  const float fxl = (float)(px - bx) + 0.5f, fyl0 = (float)(py0 - by) + 0.5f, fyl1 = fyl0 + 1.f;
  uint2 rg = ranges[tile];
  if (!in_bounds(rg.x <= rg.y && rg.y <= b.cap_pairs, b.flags)) rg = make_uint2(0u, 0u);
  const float a_min = b.p.alpha_min, a_max = b.p.alpha_max, t_min = b.p.t_min;
  PixF P0{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, rg.y, !(px < v.W && py0 < v.H)};
  PixF P1{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, rg.y, !(px < v.W && py0 + 1 < v.H)};
  for (uint32_t start = rg.x; start < rg.y; start += NB) {
    if (__syncthreads_count(!(P0.done && P1.done)) == 0) break;
#pragma unroll
    for (int h = 0; h < NB / NT; ++h) {
      const uint32_t jj = start + threadIdx.x + h * NT;
      if (jj < rg.y) {
        const uint32_t g = pair_g[jj];
        if (in_bounds(g < b.cap_g, b.flags)) stage_record(s, threadIdx.x + h * NT, rec, g, a_min, ox, oy);
      }
    }
    __syncthreads();
    const int cnt = min((uint32_t)NB, rg.y - start);
    for (int k = 0; k < cnt; ++k) {
      if ((k & 3) == 0 && __all_sync(0xffffffffu, P0.done && P1.done)) break;
      const float4 q = s.q[k];
      const float2 m = s.m[k];
      const float p_lo = s.n[k].w;
      const float dx = __fsub_rn(fxl, m.x);
      const float pw0 = eval_power(q, dx, __fsub_rn(fyl0, m.y));
      const float pw1 = eval_power(q, dx, __fsub_rn(fyl1, m.y));
      // skip power > 0 and alpha < alpha_min (taken on the exponent); the warp skips a record none of its pixels takes
      const bool t0 = !P0.done && !(pw0 > 0.f) && pw0 >= p_lo;
      const bool t1 = !P1.done && !(pw1 > 0.f) && pw1 >= p_lo;
      if (!__any_sync(0xffffffffu, t0 || t1)) continue;
      const float4 c = s.c[k], nn = s.n[k];
      const uint32_t j = start + k;
      fwd_take<STATS>(P0, t0, pw0, q.w, c, nn, j, a_max, t_min);
      fwd_take<STATS>(P1, t1, pw1, q.w, c, nn, j, a_max, t_min);
    }
  }
  fwd_write(P0, v, b.p, px, py0, rg.x, out, b.total_pixels, b.flags);
  fwd_write(P1, v, b.p, px, py0 + 1, rg.x, out, b.total_pixels, b.flags);
}

struct PixB {            // backward state of one pixel
  float fy, T;
  float gC0, gC1, gC2, gD, gN0, gN1, gN2;       // dL/d(colour, D, N) at the pixel
  float GS;     // sum over channels of g_ch * (suffix sum of the later contributors' channel values)
  uint32_t last;
};

__device__ __forceinline__ void bwd_setup(PixB& P, const ViewDev& v, const ParamsDev& p, int px, int py, float fx_rel,
                                          const pgs_image_ptrs& img, const pgs_image_grad_ptrs& gi,
                                          long long total_pixels, uint32_t* flags) {
  P.fy = (float)py + 0.5f - v.cy;
  P.T = 1.f; P.last = 0;
  P.gC0 = P.gC1 = P.gC2 = P.gD = P.gN0 = P.gN1 = P.gN2 = 0.f;
  P.GS = 0.f;
  if (px >= v.W || py >= v.H) return;
  const long long HW = (long long)v.W * v.H;
  const long long q = v.pix_off + (long long)py * v.W + px;
  const long long q3 = 3 * v.pix_off + (long long)py * v.W + px;
  if (!in_bounds(q < total_pixels, flags)) return;
  P.last = img.last[q];
  P.T = img.t_final[q];
  P.gC0 = gi.rgb[q3]; P.gC1 = gi.rgb[q3 + HW]; P.gC2 = gi.rgb[q3 + 2 * HW];
  P.gN0 = gi.normal[q3]; P.gN1 = gi.normal[q3 + HW]; P.gN2 = gi.normal[q3 + 2 * HW];
  // chain through D_hat = D / (N . r)
  const float gDh = gi.depth[q];
  const float N0 = img.normal[q3], N1 = img.normal[q3 + HW], N2 = img.normal[q3 + 2 * HW];
  const float rx = fx_rel / v.fx, ry = P.fy / v.fy;
  const float ndr = N0 * rx + N1 * ry + N2;
  const bool ok = fabsf(ndr) >= 1e-8f && (1.f - P.T) >= 1e-6f;
  if (ok) {
    const float D = img.dist[q];
    const float ind = 1.f / ndr;
    P.gD = gDh * ind;
    const float k = -gDh * D * ind * ind;
    P.gN0 += k * rx; P.gN1 += k * ry; P.gN2 += k;
  }
  // the background enters the RGB suffix sums with weight T_final
  P.GS = P.T * p.bg * (P.gC0 + P.gC1 + P.gC2);
}

// Per-Gaussian gradients from the reduced sums: power_nat = -1/2 (A dx^2 + 2B dx dy + C dy^2)
// with dx = px - mx, so d/dmx = A dx + B dy, d/dA = -1/2 dx^2, d/dB = -dx dy, d/dC = -1/2 dy^2,
// and d alpha / d o = alpha_raw / o.
__device__ __forceinline__ void finish_grads(const float* a, float4 q, float out[13]) {
  const float An = q.x * (1.f / kHalfLog2e), Bn = q.y * (1.f / kNegLog2e), Cn = q.z * (1.f / kHalfLog2e);
  out[0] = An * a[0] + Bn * a[1];
  out[1] = Bn * a[0] + Cn * a[1];
  out[2] = -0.5f * a[2];
  out[3] = -a[3];
  out[4] = -0.5f * a[4];
  out[5] = a[5] / q.w;
#pragma unroll
  for (int f = 6; f < 13; ++f) out[f] = a[f];
}

// Backward, record-parallel within the tile: one warp per tile.  The tile's
// list is taken back to front in chunks of up to 32 records held by each of two
// 16-lane groups (two records per lane; chunks of up to 16, one record per lane,
// in 2 or 4 groups).  The pixels that still have contributors at or below the
// chunk's top (last > cbase) are split between the groups, and within a group
// stream through the lanes from the top lane down to lane 0, one lane per step,
// so each pixel meets the chunk's records in descending order as the reverse
// pass requires.  A pixel's running state (T, GS) moves down one lane per step
// by shuffle and is parked in shared memory between chunks.  Each lane sums its
// own records' per-pixel terms in registers (no reduction per pixel), the groups'
// sums are added once per chunk, and each record's gradient goes to global
// memory once per (record, tile).
//   acc[0..5]  = sum G dx, G dy, G dx^2, G dx dy, G dy^2, G   (G = dL/dalpha * alpha_raw)
//   acc[6..12] = sum w gC (3), w gD, w gN (3)
// dL/dalpha_i = T_i (g . f_i) - (g . S_i) / (1 - alpha_i), with g . S_i carried as one scalar GS.
constexpr int kBwdWarps = 2;     // warps per CTA, each on its own tile
constexpr int kTilePix = 256;

struct BwdTab {                  // per pixel of the tile, in pixel order
  float4 g0[kTilePix];           // dL/dC (3), dL/dD
  float4 g1[kTilePix];           // dL/dN (3), last contributor + 1 (bits)
  float2 f[kTilePix];            // pixel centre relative to the block origin
  float2 st[kTilePix];           // running (T, GS)
  uint8_t live[kTilePix];        // pixels still live in the current chunk
};

// One record of a lane against the pixel passing through it: undo the
// record's contribution to the pixel's transmittance (T_i = T_{i+1} / (1 - alpha_i)),
// carry GS, and add the pixel's terms to the record's sums.  Branch-free: a
// pair that the forward did not take leaves T, GS and the sums unchanged.
__device__ __forceinline__ void bwd_pair(const RecF& r, float2 mt, uint32_t j, bool act, const float4 g0,
                                         const float4 g1, const float2 f, float& T, float& GS,
                                         float acc[kGradFields], float a_max) {
  const float dx = __fsub_rn(f.x, mt.x), dy = __fsub_rn(f.y, mt.y);
  const float xx = __fmul_rn(dx, dx), xy = __fmul_rn(dx, dy), yy = __fmul_rn(dy, dy);
  const float power = eval_power_xy(r.q, xx, xy, yy);
  const bool take = act && j < __float_as_uint(g1.w) && !(power > 0.f) && power >= r.n.w;
  const float a_raw = __fmul_rn(r.q.w, ex2_approx(power));
  const float alpha = fminf(a_max, a_raw);
  const float iom = rcp_approx(__fsub_rn(1.f, alpha));
  const float Tin = T, GSin = GS;
  T = take ? Tin * iom : Tin;
  const float w = take ? alpha * T : 0.f;
  float gf = g0.x * r.c.x;
  gf = fmaf(g0.y, r.c.y, gf); gf = fmaf(g0.z, r.c.z, gf); gf = fmaf(g0.w, r.c.w, gf);
  gf = fmaf(g1.x, r.n.x, gf); gf = fmaf(g1.y, r.n.y, gf); gf = fmaf(g1.z, r.n.z, gf);
  const float dLda = fmaf(T, gf, -GSin * iom);
  GS = fmaf(w, gf, GSin);
  acc[6] = fmaf(w, g0.x, acc[6]); acc[7] = fmaf(w, g0.y, acc[7]); acc[8] = fmaf(w, g0.z, acc[8]);
  acc[9] = fmaf(w, g0.w, acc[9]);
  acc[10] = fmaf(w, g1.x, acc[10]); acc[11] = fmaf(w, g1.y, acc[11]); acc[12] = fmaf(w, g1.z, acc[12]);
  // alpha clamped at alpha_max carries no gradient to o, mean, conic
  const float G = (take && !(a_raw > a_max)) ? dLda * a_raw : 0.f;
  acc[0] = fmaf(G, dx, acc[0]);
  acc[1] = fmaf(G, dy, acc[1]);
  acc[2] = fmaf(G, xx, acc[2]);
  acc[3] = fmaf(G, xy, acc[3]);
  acc[4] = fmaf(G, yy, acc[4]);
  acc[5] += G;
}

// The two records A (list index jA = jB + 1, met first on the way down) and B
// of a lane, packed half by half (A low, B high) for the f32x2 pair step.
struct RecPair {
  f2 mx, my, qx, qy, qz, qw, c0, c1, c2, c3, n0, n1, n2;
  float ploA, ploB;
};
__device__ __forceinline__ RecPair pack_records(const RecF& a, float2 ma, const RecF& b, float2 mb) {
  RecPair R;
  R.mx = f2_make(ma.x, mb.x); R.my = f2_make(ma.y, mb.y);
  R.qx = f2_make(a.q.x, b.q.x); R.qy = f2_make(a.q.y, b.q.y); R.qz = f2_make(a.q.z, b.q.z);
  R.qw = f2_make(a.q.w, b.q.w);
  R.c0 = f2_make(a.c.x, b.c.x); R.c1 = f2_make(a.c.y, b.c.y); R.c2 = f2_make(a.c.z, b.c.z);
  R.c3 = f2_make(a.c.w, b.c.w);
  R.n0 = f2_make(a.n.x, b.n.x); R.n1 = f2_make(a.n.y, b.n.y); R.n2 = f2_make(a.n.z, b.n.z);
  R.ploA = a.n.w; R.ploB = b.n.w;
  return R;
}

// bwd_pair for records A then B at one pixel, with every operation that does
// not depend on the other record done on both halves at once (f32x2, each half
// rounded as the scalar form, so alphas are the forward's bit for bit); the
// transmittance and GS chain stays scalar (B sees A's update).
__device__ __forceinline__ void bwd_pair2(const RecPair& R, uint32_t jA, uint32_t jB, bool actA, bool actB,
                                          const float4 g0, const float4 g1, const float2 f, float& T, float& GS,
                                          f2 (&acc)[kGradFields], float a_max) {
  const f2 dx = f2_sub(f2_splat(f.x), R.mx), dy = f2_sub(f2_splat(f.y), R.my);
  const f2 xx = f2_mul(dx, dx), xy = f2_mul(dx, dy), yy = f2_mul(dy, dy);
  const f2 pw = f2_fma(R.qx, xx, f2_fma(R.qz, yy, f2_mul(R.qy, xy)));
  const float pA = f2_lo(pw), pB = f2_hi(pw);
  const uint32_t last = __float_as_uint(g1.w);
  const bool tA = actA && jA < last && !(pA > 0.f) && pA >= R.ploA;
  const bool tB = actB && jB < last && !(pB > 0.f) && pB >= R.ploB;
  const f2 araw = f2_mul(R.qw, f2_make(ex2_approx(pA), ex2_approx(pB)));
  const float arA = f2_lo(araw), arB = f2_hi(araw);
  const float alA = fminf(a_max, arA), alB = fminf(a_max, arB);
  const f2 om = f2_sub(f2_splat(1.f), f2_make(alA, alB));
  const float iomA = rcp_approx(f2_lo(om)), iomB = rcp_approx(f2_hi(om));
  f2 gf = f2_mul(f2_splat(g0.x), R.c0);
  gf = f2_fma(f2_splat(g0.y), R.c1, gf); gf = f2_fma(f2_splat(g0.z), R.c2, gf); gf = f2_fma(f2_splat(g0.w), R.c3, gf);
  gf = f2_fma(f2_splat(g1.x), R.n0, gf); gf = f2_fma(f2_splat(g1.y), R.n1, gf); gf = f2_fma(f2_splat(g1.z), R.n2, gf);
  const float gfA = f2_lo(gf), gfB = f2_hi(gf);
  const float T1 = tA ? T * iomA : T;
  const float wA = tA ? alA * T1 : 0.f;
  const float dA = fmaf(T1, gfA, -GS * iomA);
  const float GS1 = fmaf(wA, gfA, GS);
  const float T2 = tB ? T1 * iomB : T1;
  const float wB = tB ? alB * T2 : 0.f;
  const float dB = fmaf(T2, gfB, -GS1 * iomB);
  GS = fmaf(wB, gfB, GS1);
  T = T2;
  const f2 w = f2_make(wA, wB);
  acc[6] = f2_fma(w, f2_splat(g0.x), acc[6]); acc[7] = f2_fma(w, f2_splat(g0.y), acc[7]);
  acc[8] = f2_fma(w, f2_splat(g0.z), acc[8]); acc[9] = f2_fma(w, f2_splat(g0.w), acc[9]);
  acc[10] = f2_fma(w, f2_splat(g1.x), acc[10]); acc[11] = f2_fma(w, f2_splat(g1.y), acc[11]);
  acc[12] = f2_fma(w, f2_splat(g1.z), acc[12]);
  // alpha clamped at alpha_max carries no gradient to o, mean, conic
  const float GA = (tA && !(arA > a_max)) ? dA * arA : 0.f;
  const float GB = (tB && !(arB > a_max)) ? dB * arB : 0.f;
  const f2 G = f2_make(GA, GB);
  acc[0] = f2_fma(G, dx, acc[0]); acc[1] = f2_fma(G, dy, acc[1]); acc[2] = f2_fma(G, xx, acc[2]);
  acc[3] = f2_fma(G, xy, acc[3]); acc[4] = f2_fma(G, yy, acc[4]); acc[5] = f2_add(acc[5], G);
}

// add one record's per-tile sums to its gradient row (nonzero float4 parts only)
__device__ __forceinline__ void flush_record(const float acc[kGradFields], float4 q, uint32_t gid,
                                             float* __restrict__ grad) {
  float a[kGradFields];
  finish_grads(acc, q, a);
  float4* dst = reinterpret_cast<float4*>(grad + (size_t)gid * 16);
  const float4 v0 = make_float4(a[0], a[1], a[2], a[3]);
  const float4 v1 = make_float4(a[4], a[5], a[6], a[7]);
  const float4 v2 = make_float4(a[8], a[9], a[10], a[11]);
  if (v0.x != 0.f || v0.y != 0.f || v0.z != 0.f || v0.w != 0.f) atomicAdd(dst, v0);
  if (v1.x != 0.f || v1.y != 0.f || v1.z != 0.f || v1.w != 0.f) atomicAdd(dst + 1, v1);
  if (v2.x != 0.f || v2.y != 0.f || v2.z != 0.f || v2.w != 0.f) atomicAdd(dst + 2, v2);
  if (a[12] != 0.f) atomicAdd(reinterpret_cast<float*>(dst + 3), a[12]);
}

// pixels with a contributor at or below index cbase, listed in pixel order; returns their number
__device__ __forceinline__ int build_live(BwdTab& tab, uint32_t cbase, int lane) {
  int n_live = 0;
#pragma unroll
  for (int p0 = 0; p0 < kTilePix; p0 += 32) {
    const bool lv = __float_as_uint(tab.g1[p0 + lane].w) > cbase;
    const unsigned m = __ballot_sync(0xffffffffu, lv);
    if (lv) tab.live[n_live + __popc(m & ((1u << lane) - 1u))] = (uint8_t)(p0 + lane);
    n_live += __popc(m);
  }
  return n_live;
}

template <int TW>
__device__ __forceinline__ void blend_bwd_tile(const BatchDev& b, int tile, BwdTab& tab,
                                               const float4* __restrict__ rec, const uint32_t* __restrict__ pair_g,
                                               const uint2* __restrict__ ranges, const pgs_image_ptrs& img,
                                               const pgs_image_grad_ptrs& gi, float* __restrict__ grad) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int TH = kTilePix / TW;
  const int lane = threadIdx.x & 31;
  const uint2 rg = ranges[tile];
  if (rg.y <= rg.x) return;
  if (!in_bounds(rg.y <= b.cap_pairs, b.flags)) return;
  const int vi = view_of_tile(b, tile);
  const ViewDev& v = b.v[vi];
  const int lt = tile - v.tile_base;
  const int ty = lt / v.tiles_x, tx = lt - ty * v.tiles_x;
  const float a_min = b.p.alpha_min, a_max = b.p.alpha_max;
  const int bx = block_origin(tx * TW), by = block_origin(ty * TH);
  const float ox = __fsub_rn((float)bx, v.cx), oy = __fsub_rn((float)by, v.cy);
  uint32_t end = 0;
  for (int p = lane; p < kTilePix; p += 32) {
    const int px = tx * TW + p % TW, py = ty * TH + p / TW;
    const float fx = (float)px + 0.5f - v.cx;
    PixB P;
    bwd_setup(P, v, b.p, px, py, fx, img, gi, b.total_pixels, b.flags);
    tab.g0[p] = make_float4(P.gC0, P.gC1, P.gC2, P.gD);
    tab.g1[p] = make_float4(P.gN0, P.gN1, P.gN2, __uint_as_float(P.last));
    tab.f[p] = make_float2((float)(px - bx) + 0.5f, (float)(py - by) + 0.5f);
    tab.st[p] = make_float2(P.T, P.GS);
    end = max(end, P.last);
  }
  end = min(__reduce_max_sync(FULL, end), rg.y);   // a stale `last` never walks past the tile's list
  for (uint32_t cend = end; cend > rg.x;) {
    const uint32_t avail = cend - rg.x;
    if (avail > 16) {
      // Chunk of 17..32 records in two lane groups of 16: lane li = lane % 16 of each
      // group holds records B = cbase + li + min(li, n2) and, for li < n2, A = B + 1;
      // each group runs its own 16-lane pipeline over half of the live pixels (a pixel
      // meets A then B in each lane, from lane 15 down to lane 0), so the pipeline fill
      // is 15 steps and a pixel's top chunk holds at most 32 records; the two groups'
      // sums are added before the atomics.
      const int n_rec = (int)min(avail, 32u);
      const uint32_t cbase = cend - n_rec;
      const int n2 = n_rec - 16;
      const int li = lane & 15, grp = lane >> 4;
      __syncwarp();
      const int n_live = build_live(tab, cbase, lane);
      const int seg = (n_live + 1) >> 1;
      const int seg_lo = grp * seg, seg_hi = min(n_live, seg_lo + seg);
      const uint32_t jB = cbase + li + min(li, n2), jA = jB + 1;
      const bool hasA = li < n2;
      uint32_t gB = pair_g[jB], gA = hasA ? pair_g[jA] : 0u;
      if (!in_bounds(gB < b.cap_g && gA < b.cap_g, b.flags)) gA = gB = 0u;
      const RecF rB = load_record(rec, gB, a_min);
      RecF rA{};
      if (hasA) rA = load_record(rec, gA, a_min);
      const float2 mtB = tile_mean(rB.m, ox, oy), mtA = tile_mean(rA.m, ox, oy);
      const RecPair R = pack_records(rA, mtA, rB, mtB);
      f2 acc[kGradFields];
#pragma unroll
      for (int f = 0; f < kGradFields; ++f) acc[f] = f2_splat(0.f);
      __syncwarp();
      float T = 0.f, GS = 0.f;
      const int nsteps = seg + 15;
#pragma unroll 2
      for (int s = 0; s < nsteps; ++s) {
        const int q = s - 15 + li;             // position in this group's slice
        const int pi = seg_lo + q;
        const bool act = q >= 0 && pi < seg_hi;
        const int pix = tab.live[act ? pi : 0];
        const float4 g1 = tab.g1[pix];
        const float2 f = tab.f[pix];
        const float4 g0 = tab.g0[pix];
        T = __shfl_down_sync(FULL, T, 1, 16);
        GS = __shfl_down_sync(FULL, GS, 1, 16);
        if (li == 15) {
          const float2 t = tab.st[pix];
          T = t.x;
          GS = t.y;
        }
        bwd_pair2(R, jA, jB, act && hasA, act, g0, g1, f, T, GS, acc, a_max);
        if (act && li == 0) tab.st[pix] = make_float2(T, GS);
      }
      float accA[kGradFields], accB[kGradFields];
#pragma unroll
      for (int f = 0; f < kGradFields; ++f) {
        const f2 t = f2_add(acc[f], f2_shfl_xor(acc[f], 16));
        accA[f] = f2_lo(t);
        accB[f] = f2_hi(t);
      }
      if (grp == 0) {
        flush_record(accB, rB.q, gB, grad);
        if (hasA) flush_record(accA, rA.q, gA, grad);
      }
      cend = cbase;
      continue;
    }
    // Single chunk of up to 16 records (the tile's last): lane l of each group holds
    // record cbase + l; the chunk is replicated into 2 or 4 lane groups that take
    // separate slices of the live pixels; their sums are combined before the atomics.
    const uint32_t cbase = rg.x;
    const int n_rec = (int)avail;
    const int gsz = n_rec <= 8 ? 8 : 16;
    const int lig = lane & (gsz - 1), grp = lane / gsz;
    const int top = n_rec - 1;                 // lane (in its group) of the chunk's last record
    __syncwarp();
    const int n_live = build_live(tab, cbase, lane);
    const int ng = 32 / gsz;
    const int seg = (n_live + ng - 1) / ng;
    const int seg_lo = grp * seg, seg_hi = min(n_live, seg_lo + seg);
    const uint32_t j = cbase + lig;
    const bool has = lig <= top;
    uint32_t gid = 0;
    RecF r{};
    if (has) {
      gid = pair_g[j];
      if (!in_bounds(gid < b.cap_g, b.flags)) gid = 0u;
      r = load_record(rec, gid, a_min);
    }
    const float2 mt = tile_mean(r.m, ox, oy);
    float acc[kGradFields];
#pragma unroll
    for (int f = 0; f < kGradFields; ++f) acc[f] = 0.f;
    __syncwarp();
    float T = 0.f, GS = 0.f;
    const int nsteps = seg + top;
#pragma unroll 2
    for (int s = 0; s < nsteps; ++s) {
      const int q = s - top + lig;             // position in this group's slice
      const int pi = seg_lo + q;
      const bool act = has && q >= 0 && pi < seg_hi;
      const int pix = tab.live[act ? pi : 0];
      const float4 g1 = tab.g1[pix];
      const float2 f = tab.f[pix];
      const float4 g0 = tab.g0[pix];
      T = __shfl_down_sync(FULL, T, 1);
      GS = __shfl_down_sync(FULL, GS, 1);
      if (lig == top) {
        const float2 t = tab.st[pix];
        T = t.x;
        GS = t.y;
      }
      bwd_pair(r, mt, j, act, g0, g1, f, T, GS, acc, a_max);
      if (act && lig == 0) tab.st[pix] = make_float2(T, GS);
    }
    for (int off = 16; off >= gsz; off >>= 1) {
#pragma unroll
      for (int f = 0; f < kGradFields; ++f) acc[f] += __shfl_xor_sync(FULL, acc[f], off);
    }
    if (has && grp == 0) flush_record(acc, r.q, gid, grad);
    cend = cbase;
  }
}

// Persistent kernels: one resident wave of CTAs takes tiles from a global queue
// in the given order (longest lists first), so long tiles do not form a tail.
template <int TW, int TH, int NB, bool STATS>
__global__ void __launch_bounds__(TW * TH / 2) k_blend_fwd(const __grid_constant__ BatchDev b,
                                                           const float4* __restrict__ rec,
                                                           const uint32_t* __restrict__ pair_g,
                                                           const uint2* __restrict__ ranges, pgs_image_ptrs out,
                                                           const uint32_t* __restrict__ order,
                                                           uint32_t* __restrict__ counter) {
  __shared__ BlendSmem<NB> s;
  __shared__ uint32_t s_next;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t it = s_next;
    if (it >= (uint32_t)b.total_tiles) break;
    const uint32_t tile = order[it];
    if (!in_bounds(tile < (uint32_t)b.total_tiles, b.flags)) continue;
    blend_fwd_tile<TW, TH, NB, STATS>(b, (int)tile, s, rec, pair_g, ranges, out);
  }
}

// Backward: every warp takes its own tiles from the queue.
template <int TW>
__global__ void __launch_bounds__(32 * kBwdWarps) k_blend_bwd(const __grid_constant__ BatchDev b,
                                                             const float4* __restrict__ rec,
                                                             const uint32_t* __restrict__ pair_g,
                                                             const uint2* __restrict__ ranges, pgs_image_ptrs img,
                                                             pgs_image_grad_ptrs gi, float* __restrict__ grad,
                                                             const uint32_t* __restrict__ order,
                                                             uint32_t* __restrict__ counter) {
  __shared__ BwdTab tabs[kBwdWarps];
  BwdTab& tab = tabs[threadIdx.x >> 5];
  for (;;) {
    uint32_t it = 0;
    if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (uint32_t)b.total_tiles) break;
    const uint32_t tile = order[it];
    if (!in_bounds(tile < (uint32_t)b.total_tiles, b.flags)) continue;
    blend_bwd_tile<TW>(b, (int)tile, tab, rec, pair_g, ranges, img, gi, grad);
  }
}

// one resident wave on the current device: SMs x CTAs per SM (both cached per device)
template <int TW, int TH, int NB, bool BWD, typename K>
static int resident_grid(K kernel, int threads, int total) {
  const int per_sm = resident_ctas_per_sm(reinterpret_cast<const void*>(kernel), threads);
  return std::max(1, std::min(total, per_sm * device_sm_count()));
}

template <int TW, int TH, int NB>
static void launch_fwd_t(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                         const pgs_image_ptrs& o, const uint32_t* order, uint32_t* ctr, cudaStream_t st) {
  if (o.n_contrib || o.n_eval) {
    const int grid = resident_grid<TW, TH, 2 * NB + 1, false>(k_blend_fwd<TW, TH, NB, true>, TW * TH / 2, b.total_tiles);
    k_blend_fwd<TW, TH, NB, true><<<grid, TW * TH / 2, 0, st>>>(b, rec, pg, rg, o, order, ctr);
  } else {
    const int grid = resident_grid<TW, TH, 2 * NB, false>(k_blend_fwd<TW, TH, NB, false>, TW * TH / 2, b.total_tiles);
    k_blend_fwd<TW, TH, NB, false><<<grid, TW * TH / 2, 0, st>>>(b, rec, pg, rg, o, order, ctr);
  }
}
template <int TW, int TH>
static bool launch_fwd_nb(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                          const pgs_image_ptrs& o, const uint32_t* order, uint32_t* ctr, cudaStream_t st) {
  switch (b.p.blend_batch) {
    case 128: launch_fwd_t<TW, TH, 128>(b, rec, pg, rg, o, order, ctr, st); return true;
    case 256: launch_fwd_t<TW, TH, 256>(b, rec, pg, rg, o, order, ctr, st); return true;
    case 512: launch_fwd_t<TW, TH, 512>(b, rec, pg, rg, o, order, ctr, st); return true;
    default: return false;
  }
}
template <int TW, int TH>
static void launch_bwd_t(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                         const pgs_image_ptrs& img, const pgs_image_grad_ptrs& gi, float* grad, const uint32_t* order,
                         uint32_t* ctr, cudaStream_t st) {
  static_assert(TW * TH == kTilePix, "256-pixel tiles");
  const int grid = resident_grid<TW, TH, 0, true>(k_blend_bwd<TW>, 32 * kBwdWarps,
                                              (b.total_tiles + kBwdWarps - 1) / kBwdWarps);
  k_blend_bwd<TW><<<grid, 32 * kBwdWarps, 0, st>>>(b, rec, pg, rg, img, gi, grad, order, ctr);
}

bool launch_blend_fwd(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                      const pgs_image_ptrs& o, const uint32_t* order, uint32_t* ctr, cudaStream_t st) {
  const int tw = b.p.tile_w, th = b.p.tile_h;
  if (tw == 16 && th == 16) return launch_fwd_nb<16, 16>(b, rec, pg, rg, o, order, ctr, st);
  if (tw == 8 && th == 32) return launch_fwd_nb<8, 32>(b, rec, pg, rg, o, order, ctr, st);
  if (tw == 32 && th == 8) return launch_fwd_nb<32, 8>(b, rec, pg, rg, o, order, ctr, st);
  return false;
}

bool launch_blend_bwd(const BatchDev& b, const float4* rec, const uint32_t* pg, const uint2* rg,
                      const pgs_image_ptrs& img, const pgs_image_grad_ptrs& gi, float* grad, const uint32_t* order,
                      uint32_t* ctr, cudaStream_t st) {
  const int tw = b.p.tile_w, th = b.p.tile_h;
  if (tw == 16 && th == 16) launch_bwd_t<16, 16>(b, rec, pg, rg, img, gi, grad, order, ctr, st);
  else if (tw == 8 && th == 32) launch_bwd_t<8, 32>(b, rec, pg, rg, img, gi, grad, order, ctr, st);
  else if (tw == 32 && th == 8) launch_bwd_t<32, 8>(b, rec, pg, rg, img, gi, grad, order, ctr, st);
  else return false;
  return true;
}

// Queue order of the tiles: descending list length (ties keep tile order), as a
// 16-bit key (two sort passes); lists of 65,535 pairs or more share the first place.
__global__ void k_tile_order_keys(const uint2* __restrict__ ranges, int n_tiles, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
    const uint2 r = ranges[t];
    const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
    keys[t] = 0xffffu - min(len, 0xffffu);
    vals[t] = (uint32_t)t;
  }
}

}  // namespace pgs
