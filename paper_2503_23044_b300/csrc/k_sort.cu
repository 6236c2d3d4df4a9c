// Binning and ordering: the reorder pi of Eq. 5 as a stable sort of
// (Gaussian-view, tile) pairs by (view tile, view depth, Gaussian index).
//
// Done as one LSD radix sort split in two stages: the depth digits are sorted
// first on the G Gaussian-views (each appears once), then every Gaussian's
// tiles are emitted in depth order and the pairs are stably sorted by tile id
// only.  Both stages use the same onesweep pass (global digit histogram once,
// then one pass per 8-bit digit with a decoupled look-back across tiles of
// 4096 keys).  Every spin in the look-back is bounded: past the limit the pass
// raises PGS_ERR_TIMEOUT and carries on, so no launch can hang.
#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace pgs {

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned long long block_exclusive_scan_u64(unsigned long long x,
                                                                       unsigned long long* s_w,
                                                                       unsigned long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < nw ? s_w[lane] : 0ull;
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) s_w[lane] = wi - w;
    if (lane == nw - 1) s_w[32] = wi;
  }
  __syncthreads();
  unsigned long long r = s_w[warp] + inc - x;
  total = s_w[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void scan_range(long long n, long long& start, long long& end) {
  const long long per = ((n + gridDim.x - 1) / gridDim.x + kScanChunk - 1) / kScanChunk * kScanChunk;
  start = min(n, (long long)blockIdx.x * per);
  end = min(n, start + per);
}

__device__ __forceinline__ uint32_t scan_in(const uint32_t* in, const uint32_t* index, long long k) {
  return index ? in[index[k]] : in[k];
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              const uint32_t* __restrict__ index,
                                                              const long long* __restrict__ d_n,
                                                              unsigned long long* __restrict__ sums) {
  __shared__ unsigned long long s_w[33];
  long long s, e;
  scan_range(*d_n, s, e);
  unsigned long long acc = 0;
  for (long long k = s + threadIdx.x; k < e; k += blockDim.x) acc += scan_in(in, index, k);
  unsigned long long tot;
  block_exclusive_scan_u64(acc, s_w, tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_spine(unsigned long long* __restrict__ sums, int nb,
                                                     unsigned long long* __restrict__ total) {
  __shared__ unsigned long long s_w[33];
  unsigned long long x = threadIdx.x < nb ? sums[threadIdx.x] : 0ull;
  unsigned long long tot;
  unsigned long long ex = block_exclusive_scan_u64(x, s_w, tot);
  if (threadIdx.x < nb) sums[threadIdx.x] = ex;
  if (threadIdx.x == 0) *total = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* __restrict__ in,
                                                            const uint32_t* __restrict__ index,
                                                            uint32_t* __restrict__ out,
                                                            const long long* __restrict__ d_n,
                                                            const unsigned long long* __restrict__ sums) {
  __shared__ unsigned long long s_w[33];
  long long s, e;
  scan_range(*d_n, s, e);
  unsigned long long carry = sums[blockIdx.x];
  for (long long c = s; c < e; c += kScanChunk) {
    uint32_t v[kScanItems];
    unsigned long long loc = 0;
    const long long b0 = c + (long long)threadIdx.x * kScanItems;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const long long k = b0 + i;
      v[i] = k < e ? scan_in(in, index, k) : 0u;
      loc += v[i];
    }
    unsigned long long tot;
    unsigned long long ex = block_exclusive_scan_u64(loc, s_w, tot) + carry;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const long long k = b0 + i;
      if (k < e) out[k] = (uint32_t)ex;
      ex += v[i];
    }
    carry += tot;
  }
}

void launch_exclusive_scan(const uint32_t* in, const uint32_t* index, uint32_t* out, unsigned long long* total,
                           const long long* d_n, unsigned long long* sums, cudaStream_t st) {
  k_scan_reduce<<<kScanBlocks, kScanThreads, 0, st>>>(in, index, d_n, sums);
  k_scan_spine<<<1, 1024, 0, st>>>(sums, kScanBlocks, total);
  k_scan_down<<<kScanBlocks, kScanThreads, 0, st>>>(in, index, out, d_n, sums);
}

// ------------------------------------------------------------------ onesweep radix sort
constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 keys per tile
static_assert(kSortTile == kSortTileKeys, "tile size shared with the scratch layout");
constexpr int kRadix = 256;          // digits of the 8-bit passes
constexpr int kRadixMax = 512;       // digits of the 9-bit passes (ranges of 17-18 or 25-27 bits)
constexpr uint32_t kStFlagAgg = 1u << 30, kStFlagInc = 2u << 30, kStMask = (1u << 30) - 1;

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// the last digit of a bit range that is not a multiple of the digit width is narrower
__host__ __device__ __forceinline__ uint32_t digit_mask(int shift, int bit_hi, int rb = 8) {
  const int w = bit_hi - shift < rb ? bit_hi - shift : rb;
  return (1u << w) - 1u;
}

SortScratch sort_scratch_layout(void* base, long long n_max, int radix_bits_max) {
  SortScratch s;
  char* p = static_cast<char*>(base);
  s.hist = reinterpret_cast<uint32_t*>(p);                 // [4][256] or [2][512]
  s.counters = s.hist + 4 * kRadix;                         // [4]
  s.err = s.counters + 4;                                   // [1] (+3 pad)
  s.max_tiles = (n_max + kSortTile - 1) / kSortTile + 1;
  s.status = s.err + 4;                                     // [2][max_tiles][256 or 512]
  s.radix_bits_max = radix_bits_max;
  s.bytes = sort_scratch_bytes_for(n_max, radix_bits_max);
  return s;
}

constexpr int kHistLoads = 8;
template <int RB>
__global__ void __launch_bounds__(256) k_sort_hist(const uint32_t* __restrict__ keys, const long long* __restrict__ d_n,
                                                   long long n_max, int bit_lo, int bit_hi, int n_pass,
                                                   uint32_t* __restrict__ hist, uint32_t* __restrict__ status0,
                                                   uint32_t* err) {
  constexpr int R = 1 << RB;
  __shared__ uint32_t s_h[4 * kRadix];                      // [n_pass][R], n_pass * R <= 1024
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) s_h[i] = 0;
  __syncthreads();
  const long long n = max(0ll, min(*d_n, n_max));
  // kHistLoads keys per thread are loaded before any of them is counted, so each thread
  // keeps that many loads in flight (counts are integers: the order of the adds is free)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; k0 < n; k0 += kHistLoads * stride) {
    uint32_t kk[kHistLoads];
#pragma unroll
    for (int u = 0; u < kHistLoads; ++u) kk[u] = k0 + u * stride < n ? keys[k0 + u * stride] : 0u;
#pragma unroll
    for (int u = 0; u < kHistLoads; ++u) {
      if (k0 + u * stride >= n) break;
      for (int p = 0; p < n_pass; ++p) {
        const int sh = bit_lo + RB * p;
        const uint32_t i = p * R + ((kk[u] >> sh) & digit_mask(sh, bit_hi, RB));
        if (in_bounds(i < 4u * kRadix, err)) atomicAdd(&s_h[i], 1u);
      }
    }
  }
  // clear the look-back status of the first pass for the live tiles
  const long long n_tiles = (n + kSortTile - 1) / kSortTile;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_tiles * R;
       k += (long long)gridDim.x * blockDim.x)
    status0[k] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n_pass * R; i += blockDim.x) {
    const uint32_t c = s_h[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// exclusive scan of each pass's digit counts: launched with R threads
template <int RB>
__global__ void __launch_bounds__(1 << RB) k_sort_hist_scan(uint32_t* __restrict__ hist, int n_pass) {
  constexpr int R = 1 << RB;
  __shared__ unsigned long long s_w[33];
  for (int p = 0; p < n_pass; ++p) {
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan_u64(hist[p * R + threadIdx.x], s_w, tot);
    hist[p * R + threadIdx.x] = (uint32_t)ex;
  }
}

// the lanes of `valid` whose RB-bit digit equals this lane's: one ballot per digit bit
// (warp-collective: every lane of the warp must call it, outside any per-lane condition)
template <int RB>
__device__ __forceinline__ uint32_t digit_peers(uint32_t dg, uint32_t valid) {
  uint32_t peers = valid;
#pragma unroll
  for (int bit = 0; bit < RB; ++bit) {
    const uint32_t bv = __ballot_sync(0xffffffffu, (dg >> bit) & 1u);
    peers &= ~(bv ^ (0u - ((dg >> bit) & 1u)));
  }
  return peers;
}

// One onesweep pass: 512 threads (two CTAs per SM) rank a tile of 4096 keys.
// Larger tiles halve the tiles in flight against 2048-key tiles, and with them the
// length of the look-back walks (about forty predecessors per digit and tile at
// 2048 keys on the 14M-pair tile sort).  The eight peer masks of a warp are
// formed first, then the per-warp running counts (16-bit: at most 4096) are
// taken in item order, which keeps the ranking stable.  Keys and values
// are reordered through dynamic shared memory (32 KB).
template <int RB>
__global__ void __launch_bounds__(kSortThreads, 2) k_sort_pass(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const long long* __restrict__ d_n, long long n_max, int shift, uint32_t dmask,
    const uint32_t* __restrict__ digit_off, uint32_t* __restrict__ counter, uint32_t* __restrict__ status,
    uint32_t* __restrict__ status_next, uint32_t* __restrict__ err, uint32_t spin_limit, uint32_t hold_tile) {
  constexpr int R = 1 << RB;   // digits: one per thread t < R
  static_assert(R <= kSortThreads, "one digit per thread");
  extern __shared__ uint32_t s_dyn[];
  uint32_t* s_keys = s_dyn;
  uint32_t* s_vals = s_dyn + kSortTile;
  __shared__ uint16_t s_whist[kSortWarps][R];
  __shared__ uint32_t s_excl[R];
  __shared__ uint32_t s_gbase[R];
  __shared__ unsigned long long s_w[33];
  __shared__ uint32_t s_tile;
  const long long n = max(0ll, min(*d_n, n_max));
  const long long n_tiles = (n + kSortTile - 1) / kSortTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const bool top_pass = status_next == nullptr;        // the last pass has no next status to clear
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
    for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= n_tiles) break;
    const long long base = tile * kSortTile + warp * (kSortTile / kSortWarps);
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      const long long idx = base + i * 32 + lane;
      const bool ok = idx < n;
      key[i] = ok ? kin[idx] : 0xffffffffu;
      val[i] = ok ? vin[idx] : 0u;
    }
    // warp-level stable ranking, item order (i, lane).  The lanes holding the same digit
    // (padding lanes match no one) come from one ballot per digit bit: `match.any`
    // serialises over the distinct digits of a warp, which the low digits of the tile
    // sort have many of.  In the top pass (the most significant digit, often one per
    // warp) a warp whose 32 digits agree skips the ballots.
    if (top_pass) {
#pragma unroll
      for (int i = 0; i < kSortItems; ++i) {
        const long long idx = base + i * 32 + lane;
        const uint32_t dg = (key[i] >> shift) & dmask;
        uint32_t peers = __ballot_sync(0xffffffffu, idx < n);
        if (!__all_sync(0xffffffffu, dg == __shfl_sync(0xffffffffu, dg, 0))) peers = digit_peers<RB>(dg, peers);
        rank[i] = idx < n ? peers : (1u << lane);
      }
    } else {
#pragma unroll
      for (int i = 0; i < kSortItems; ++i) {
        const long long idx = base + i * 32 + lane;
        const uint32_t dg = (key[i] >> shift) & dmask;
        const uint32_t peers = digit_peers<RB>(dg, __ballot_sync(0xffffffffu, idx < n));   // every lane votes
        rank[i] = idx < n ? peers : (1u << lane);
      }
    }
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      const long long idx = base + i * 32 + lane;
      const bool ok = idx < n;
      const uint32_t dg = (key[i] >> shift) & dmask;
      const uint32_t peers = rank[i];
      const uint32_t before = s_whist[warp][dg];
      __syncwarp();
      rank[i] = before + __popc(peers & lt_mask);
      if (ok && (peers & lt_mask) == 0) s_whist[warp][dg] = (uint16_t)(before + __popc(peers));
      __syncwarp();
    }
    __syncthreads();
    // digit d = t of the first R threads: counts of the tile (warp order kept in s_whist)
    const int d = threadIdx.x;
    const bool dthr = d < R;
    uint32_t run = 0;
    if (dthr) {
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = s_whist[w][d];
        s_whist[w][d] = (uint16_t)run;
        run += c;
      }
    }
    uint32_t* st = status + tile * R;
    // (hold_tile: a failure-path test hook; that tile never publishes, so the next one's wait runs out)
    if (dthr && tile != hold_tile) st_relaxed(st + d, (tile == 0 ? kStFlagInc : kStFlagAgg) | run);
    unsigned long long tot;
    const uint32_t excl = (uint32_t)block_exclusive_scan_u64(run, s_w, tot);
    if (dthr) {
      s_excl[d] = excl;
      // decoupled look-back over earlier tiles, eight status words per round
      // (independent loads), each wait bounded
      uint32_t prefix = 0;
      if (tile > 0) {
        long long j = tile - 1;
        uint32_t spins = 0;
        bool stop = false;
        while (!stop && j >= 0) {
          constexpr int kLB = 8;
          uint32_t w[kLB];
#pragma unroll
          for (int q = 0; q < kLB; ++q) w[q] = (j - q >= 0) ? ld_relaxed(status + (j - q) * R + d) : kStFlagInc;
#pragma unroll
          for (int q = 0; q < kLB; ++q) {
            if (stop) break;
            uint32_t f = w[q] & ~kStMask;
            while (f == 0u) {          // tile j - q has not published yet
              if (++spins > spin_limit) { atomicOr(err, kFlagTimeout); break; }
              if ((spins & 255u) == 0u && (ld_relaxed(err) & kFlagTimeout)) break;
              __nanosleep(32);
              w[q] = ld_relaxed(status + (j - q) * R + d);
              f = w[q] & ~kStMask;
            }
            if (f == 0u) { stop = true; break; }   // gave up (timeout flagged)
            if (j - q < 0) { stop = true; break; }  // ran past tile 0
            prefix += w[q] & kStMask;
            if (f == kStFlagInc) stop = true;
          }
          j -= kLB;
        }
        if (tile != hold_tile) st_relaxed(st + d, kStFlagInc | ((prefix + run) & kStMask));
      }
      s_gbase[d] = digit_off[d] + prefix - excl;
      if (status_next) status_next[tile * R + d] = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      const long long idx = base + i * 32 + lane;
      if (idx < n) {
        const uint32_t dg = (key[i] >> shift) & dmask;
        const uint32_t lp = s_excl[dg] + s_whist[warp][dg] + rank[i];
        if (in_bounds(lp < (uint32_t)kSortTile, err)) {
          s_keys[lp] = key[i];
          s_vals[lp] = val[i];
        }
      }
    }
    __syncthreads();
    const int cnt = (int)min((long long)kSortTile, n - tile * kSortTile);
    for (int j = threadIdx.x; j < cnt; j += kSortThreads) {
      const uint32_t k = s_keys[j];
      const uint32_t pos = s_gbase[(k >> shift) & dmask] + (uint32_t)j;
      if ((long long)pos < n) {   // always true unless a look-back wait ran out
        kout[pos] = k;
        vout[pos] = s_vals[j];
      }
    }
    __syncthreads();
  }
}

__global__ void k_copy_pairs(const uint32_t* __restrict__ ks, const uint32_t* __restrict__ vs, uint32_t* __restrict__ kd,
                             uint32_t* __restrict__ vd, const long long* __restrict__ d_n, long long n_max) {
  const long long n = max(0ll, min(*d_n, n_max));
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    kd[k] = ks[k];
    vd[k] = vs[k];
  }
}

// digit width of a sort: 9 bits where that saves a pass and the scratch allows it.  The histogram area
// holds 4 x 256 = 2 x 512 digit counts, so 9-bit digits are taken for two passes only (17-18 bits).
static int sort_digit_bits(int bit_lo, int bit_hi, int radix_bits_max) {
  const int bits = bit_hi - bit_lo;
  return (radix_bits_max >= 9 && bits > 16 && bits <= 18) ? 9 : 8;
}
int sort_passes(int bit_lo, int bit_hi) { return (bit_hi - bit_lo + 7) / 8; }

// After a sort whose look-back wait ran out (kFlagTimeout set) the output may
// hold stale entries; leave only indices the consumers can use safely:
// identity values (vals[i] = i, i < n) or, without vals, no items (*d_n = 0).
__global__ void k_sort_timeout_guard(const uint32_t* __restrict__ flags, long long* __restrict__ d_n, long long n_max,
                                     uint32_t* __restrict__ vals) {
  if (!(ld_relaxed(flags) & kFlagTimeout)) return;
  if (!vals) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_n = 0;
    return;
  }
  const long long n = max(0ll, min(*d_n, n_max));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    vals[i] = (uint32_t)i;
}

template <int RB>
static cudaError_t launch_sort_rb(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                  const long long* d_n, long long n_max, int bit_lo, int bit_hi, const SortScratch& s,
                                  uint32_t* err, uint32_t spin_limit, uint32_t hold_tile, int num_sms, cudaStream_t st,
                                  int* n_launch) {
  constexpr int R = 1 << RB;
  const int np = (bit_hi - bit_lo + RB - 1) / RB;
  if (n_launch) *n_launch = 0;
  if (np <= 0) return cudaSuccess;
  if (np * R > 4 * kRadix) return cudaErrorInvalidValue;   // more digit counts than the histogram area holds
  if (n_launch) *n_launch = 2 + np + (np & 1);
  cudaError_t e = cudaMemsetAsync(s.hist, 0, (size_t)(4 * kRadix + 4) * 4, st);
  if (e != cudaSuccess) return e;
  uint32_t* status[2] = {s.status, s.status + (size_t)s.max_tiles * R};
  k_sort_hist<RB><<<num_sms * 4, 256, 0, st>>>(keys, d_n, n_max, bit_lo, bit_hi, np, s.hist, status[0], err);
  k_sort_hist_scan<RB><<<1, R, 0, st>>>(s.hist, np);
  // persistent passes: one resident wave (tiles are taken from a counter)
  const size_t dsm = 2 * kSortTile * sizeof(uint32_t);
  const int per_sm = prepare_smem_kernel(reinterpret_cast<const void*>(k_sort_pass<RB>), kSortThreads, dsm);
  const int pass_grid = (int)std::max(1ll, std::min((long long)per_sm * num_sms, (n_max + kSortTile - 1) / kSortTile));
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  for (int p = 0; p < np; ++p) {
    k_sort_pass<RB><<<pass_grid, kSortThreads, dsm, st>>>(ki, vi, ko, vo, d_n, n_max, bit_lo + RB * p,
                                                        digit_mask(bit_lo + RB * p, bit_hi, RB), s.hist + p * R,
                                                        s.counters + p, status[p & 1],
                                                        p + 1 < np ? status[(p + 1) & 1] : nullptr, err, spin_limit,
                                                        hold_tile);
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  if (ki != keys) k_copy_pairs<<<num_sms * 4, 256, 0, st>>>(ki, vi, keys, vals, d_n, n_max);
  return cudaGetLastError();
}

cudaError_t launch_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                              const long long* d_n, long long n_max, int bit_lo, int bit_hi, const SortScratch& s,
                              uint32_t* err, uint32_t spin_limit, uint32_t hold_tile, int num_sms, cudaStream_t st,
                              int* n_launch) {
  if (sort_digit_bits(bit_lo, bit_hi, s.radix_bits_max) == 9)
    return launch_sort_rb<9>(keys, vals, keys_alt, vals_alt, d_n, n_max, bit_lo, bit_hi, s, err, spin_limit,
                             hold_tile, num_sms, st, n_launch);
  return launch_sort_rb<8>(keys, vals, keys_alt, vals_alt, d_n, n_max, bit_lo, bit_hi, s, err, spin_limit, hold_tile,
                           num_sms, st, n_launch);
}

// ------------------------------------------------------------------ pair emission and tile ranges
// Pair emission.  A warp takes 32 consecutive Gaussian-views in depth order;
// their output runs are adjacent (offsets are an exclusive scan in that order),
// so each lane writes its tiles into the warp's shared-memory window and the
// warp then copies the window out with coalesced stores.  Pairs past the
// window go to global memory directly.  A Gaussian with more than kEmitBig
// pairs is emitted afterwards by the whole warp, one tile row per lane.
constexpr int kEmitWarps = 4;
constexpr int kEmitStage = 1024;   // staged pairs per warp
constexpr uint32_t kEmitBig = 96;

// write pair (tid, g) at output position o of a warp whose window starts at wbase
__device__ __forceinline__ void emit_one(long long o, long long wbase, uint32_t tid, uint32_t g, long long cap,
                                         uint32_t* s_t, uint32_t* s_g, uint32_t* __restrict__ tiles_out,
                                         uint32_t* __restrict__ g_out, uint32_t* err) {
  const long long rel = o - wbase;
  if (!in_bounds(rel >= 0, err)) return;
  if (rel < kEmitStage) {
    s_t[rel] = tid;
    s_g[rel] = g;
  } else if (o < cap) {
    tiles_out[o] = tid;
    g_out[o] = g;
  }
}

__global__ void __launch_bounds__(32 * kEmitWarps) k_emit_pairs(const __grid_constant__ BatchDev b,
                                                                const float4* __restrict__ rec,
                                                                const uint32_t* __restrict__ counts,
                                                                const uint32_t* __restrict__ sorted_g,
                                                                const uint32_t* __restrict__ offs,
                                                                const long long* __restrict__ d_ng, long long cap,
                                                                int mode, long long n_explicit,
                                                                const uint32_t* __restrict__ rows,
                                                                uint32_t* __restrict__ tiles_out,
                                                                uint32_t* __restrict__ g_out, uint32_t* err) {
  __shared__ uint32_t s_t[kEmitWarps][kEmitStage];
  __shared__ uint32_t s_g[kEmitWarps][kEmitStage];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long ng = *d_ng;
  const long long stride = (long long)gridDim.x * kEmitWarps * 32;
  for (long long kb = ((long long)blockIdx.x * kEmitWarps + w) * 32; kb < ng; kb += stride) {
    const long long k = kb + lane;
    const bool ok = k < ng;
    uint32_t g = 0u, cnt = 0u;
    long long o = 0;
    if (ok) {
      g = sorted_g[k];
      if (!in_bounds(g < (uint32_t)b.cap_g, err)) g = 0u;
      cnt = counts[g];
      o = offs[k];
    }
    const long long wbase = __shfl_sync(0xffffffffu, o, 0);   // lane 0 (k = kb < ng) starts the window
    const long long o_beg = o, o_end = o + cnt;
    const bool big = cnt > kEmitBig;
    if (cnt && !big) {
      const int vi = mode == PGS_MODE_EXPLICIT ? (int)(g / n_explicit) : (int)(rows[g / kNOff] >> 27);
      const ViewDev& v = b.v[vi];
      TileEllipse e;
      const float4 r0 = rec[(long long)g * kRecF4], r1 = rec[(long long)g * kRecF4 + 1];
      if (tile_ellipse_setup(r0, r1, b.p, e)) {
        const int tb = v.tile_base, tx_n = v.tiles_x;
        for_each_tile_row(e, v, b.p.tile_w, b.p.tile_h, [&](int ty, int c0, int c1) {
          for (int tx = c0; tx <= c1; ++tx) {
            if (o < o_end) emit_one(o, wbase, (uint32_t)(tb + ty * tx_n + tx), g, cap, s_t[w], s_g[w], tiles_out, g_out, err);
            ++o;
          }
        });
      }
      if (o != o_end) set_flag(err, kFlagCapacity);   // count and emit disagree: never expected
    }
    // large Gaussians: the warp takes them one at a time, lane l on tile rows ty0 + l, ty0 + l + 32, ...
    unsigned bigs = __ballot_sync(0xffffffffu, ok && big);
    while (bigs) {
      const int src = __ffs(bigs) - 1;
      bigs &= bigs - 1u;
      const uint32_t gb = __shfl_sync(0xffffffffu, g, src);
      const long long ob = __shfl_sync(0xffffffffu, o_beg, src), oe = __shfl_sync(0xffffffffu, o_end, src);
      const int vi = mode == PGS_MODE_EXPLICIT ? (int)(gb / n_explicit) : (int)(rows[gb / kNOff] >> 27);
      const ViewDev& v = b.v[vi];
      TileEllipse e;
      const float4 r0 = rec[(long long)gb * kRecF4], r1 = rec[(long long)gb * kRecF4 + 1];
      const bool okb = tile_ellipse_setup(r0, r1, b.p, e);   // same record, same answer in every lane
      long long pos = ob;
      if (okb) {
        const TileRows R = tile_rows(e, v, b.p.tile_w, b.p.tile_h);
        const int tb = v.tile_base, tx_n = v.tiles_x;
        for (int r0w = R.ty0; r0w <= R.ty1; r0w += 32) {   // warp-uniform bounds
          const int ty = r0w + lane;
          int c0 = 0, c1 = -1;
          if (ty <= R.ty1 && !tile_row_span(e, v, b.p.tile_w, b.p.tile_h, R, ty, c0, c1)) c1 = c0 - 1;
          const uint32_t rc = (uint32_t)max(0, c1 - c0 + 1);
          uint32_t incl = rc;   // warp inclusive scan of the row counts
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
          }
          long long q = pos + (incl - rc);
          for (int tx = c0; tx <= c1; ++tx, ++q)
            if (q < oe) emit_one(q, wbase, (uint32_t)(tb + ty * tx_n + tx), gb, cap, s_t[w], s_g[w], tiles_out, g_out, err);
          pos += __shfl_sync(0xffffffffu, incl, 31);
        }
      }
      if (lane == 0 && pos != oe) set_flag(err, kFlagCapacity);   // count and emit disagree: never expected
    }
    __syncwarp();
    const uint32_t my_len = ok ? (uint32_t)(o_end - wbase) : 0u;
    const uint32_t wlen = min(__reduce_max_sync(0xffffffffu, my_len), (uint32_t)kEmitStage);
    for (uint32_t i = lane; i < wlen; i += 32) {
      const long long p = wbase + i;
      if (p < cap) {
        tiles_out[p] = s_t[w][i];
        g_out[p] = s_g[w][i];
      }
    }
    __syncwarp();
  }
}

__global__ void k_pairs_total(const unsigned long long* __restrict__ total, long long cap, long long* __restrict__ d_p,
                              uint32_t* err) {
  const unsigned long long t = *total;
  if (t > (unsigned long long)cap) set_flag(err, kFlagCapacity);
  *d_p = (long long)min(t, (unsigned long long)cap);
}

__global__ void k_tile_ranges(const uint32_t* __restrict__ tiles, const long long* __restrict__ d_p,
                              uint2* __restrict__ ranges, int n_tiles, uint32_t* err) {
  const long long P = *d_p;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t t = tiles[i];
    if (!in_bounds(t < (uint32_t)n_tiles, err)) continue;
    if (i == 0 || tiles[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == P - 1 || tiles[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

}  // namespace pgs
