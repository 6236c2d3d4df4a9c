// Shared decoder F_de (Eq. 4) on the 5th-generation tensor cores: BF16
// operands, FP32 accumulation in tensor memory, the activation / projection
// epilogue fused behind it.
//
// One CTA of 128 threads decodes 128 visible (view, anchor) rows at a time:
//   layer 1  D1[128 x 32]  = X[128 x 48] . W1^T    (inputs padded 35 -> 48)
//   layer 2  D2[128 x 160] = H[128 x 32] . W2p^T   (outputs permuted, 11 per Gaussian,
//                                                    two Gaussians per 32-column group)
// Thread t owns row t: it writes its operand row to shared memory, reads its
// accumulator row back with tcgen05.ld (warp w sees lanes 32w..32w+31) and
// runs the epilogue of its 10 Gaussians.  One elected thread issues the MMAs.
// Operands use the no-swizzle K-major core-matrix layout: 8 rows x 16 bytes
// per core matrix, K-adjacent core matrices 128 B apart (LBO), 8-row groups
// SBO apart.  Every wait on the MMA barrier is bounded; on a timeout the
// kernel raises PGS_ERR_TIMEOUT, waits once more, frees its tensor memory and
// returns.
#include <cuda_bf16.h>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"
#include "pgs_project.cuh"

namespace pgs {

namespace tc {

constexpr int kRows = 128;
constexpr int kK1 = 48, kN1 = 32;           // layer 1: K padded from 35 (or 36), N = hidden
constexpr int kK2 = 32, kN2 = 160;          // layer 2: K = hidden, N = 5 groups x 32 columns
constexpr int kGroupCols = 32, kPerGauss = 11;
constexpr uint32_t kTmemCols = 256;         // D1 at column 0, D2 at column 32
constexpr uint32_t kD2Col = 32;

struct Smem {
  __nv_bfloat16 A1[kRows * kK1];            // 12288 B
  __nv_bfloat16 B1[kN1 * kK1];              //  3072 B
  __nv_bfloat16 A2[kRows * kK2];            //  8192 B
  __nv_bfloat16 B2[kN2 * kK2];              // 10240 B
  float b1[kN1];
  float b2p[kN2];
  unsigned long long mbar;
  uint32_t tmem_base;
  int abort;
};

// byte offset of element (row r, k) in a K-major no-swizzle tile with K = kdim
__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int kdim) {
  return (uint32_t)((r >> 3) * (kdim / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start >> 4, LBO >> 4 at bit 16, SBO >> 4 at
// bit 32, descriptor version 1 at bit 46, no swizzle (layout type 0 at bit 61)
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D = F32 (bit 4), A = B = BF16 (bits 7, 10),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the MMA barrier phase
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < (1u << 22); ++i)
    if (mbar_try(mbar, parity)) return true;
  return false;
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// permuted layer-2 output column n -> original output index of Eq. 4's blocked layout, or -1 (padding)
__host__ __device__ inline int perm_out(int n) {
  const int grp = n / kGroupCols, w = n % kGroupCols;
  if (w >= 2 * kPerGauss) return -1;
  const int j = 2 * grp + w / kPerGauss, t = w % kPerGauss;
  if (t == 0) return j;
  if (t <= 3) return 10 + 3 * j + (t - 1);
  if (t <= 6) return 40 + 3 * j + (t - 4);
  return 70 + 4 * j + (t - 7);
}

}  // namespace tc

using namespace tc;

// 384 threads: warps 0-3 own rows 0-127 of a tile for the operands and layer 1
// (warp w reads TMEM lanes 32 (w mod 4) .. + 31); after layer 2, warps w, w + 4
// and w + 8 share those 32 rows, taking Gaussians 0-3, 4-6 and 7-9 of each row.
constexpr int kTcThreads = 384;
__device__ __forceinline__ int epi_first(int part) { return part == 0 ? 0 : (part == 1 ? 4 : 7); }

__global__ void __launch_bounds__(kTcThreads) k_decode_project_tc(const __grid_constant__ BatchDev b, pgs_anchor_ptrs A,
                                                           pgs_mlp_ptrs Wt, const uint32_t* __restrict__ rows,
                                                           const long long* __restrict__ n_rows_p, long long cap,
                                                           float4* __restrict__ rec, uint32_t* __restrict__ counts,
                                                           uint32_t* __restrict__ keys, DecodeOut dec, uint32_t* err) {
  __shared__ __align__(1024) Smem sm;
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool row_thread = tid < kRows;                // operand rows and layer 1
  const int erow = (warp & 3) * 32 + (tid & 31);      // the row whose Gaussians this thread projects
  const int epart = warp >> 2;                        // Gaussians epi_first(epart) .. epi_first(epart + 1) - 1
  const int in_dim = b.p.in_dim;
  char* A1b = reinterpret_cast<char*>(sm.A1);
  char* B1b = reinterpret_cast<char*>(sm.B1);
  char* A2b = reinterpret_cast<char*>(sm.A2);
  char* B2b = reinterpret_cast<char*>(sm.B2);
  // decoder weights -> BF16 operand tiles (zero padded); biases stay FP32 for the epilogue
  for (int t = tid; t < kN1 * kK1; t += kTcThreads) {
    const int n = t / kK1, k = t % kK1;
    const float w = k < in_dim ? Wt.W1[n * in_dim + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(B1b + kmaj_off(n, k, kK1)) = __float2bfloat16_rn(w);
  }
  for (int t = tid; t < kN2 * kK2; t += kTcThreads) {
    const int n = t / kK2, k = t % kK2;
    const int o = perm_out(n);
    const float w = o >= 0 ? Wt.W2[o * kHidden + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(B2b + kmaj_off(n, k, kK2)) = __float2bfloat16_rn(w);
  }
  if (tid < kN1) sm.b1[tid] = Wt.b1[tid];
  for (int t = tid; t < kN2; t += kTcThreads) {
    const int o = perm_out(t);
    sm.b2p[t] = o >= 0 ? Wt.b2[o] : 0.f;
  }
  const uint32_t mbar = smem_u32(&sm.mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.tmem_base;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t a1 = smem_u32(sm.A1), b1s = smem_u32(sm.B1), a2 = smem_u32(sm.A2), b2s = smem_u32(sm.B2);
  constexpr uint32_t kIdesc1 = make_idesc(kRows, kN1), kIdesc2 = make_idesc(kRows, kN2);
  const long long n_rows = min(*n_rows_p, cap);
  const long long n_tiles = (n_rows + kRows - 1) / kRows;
  uint32_t phase = 0;
  bool timed_out = false;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    if (row_thread) {
      const long long r = tile * kRows + tid;
      float X[kMaxIn];
#pragma unroll
      for (int k = 0; k < kMaxIn; ++k) X[k] = 0.f;
      if (r < n_rows) {
        const uint32_t rw = rows[r];
        decoder_input(A, b.v[rw >> 27], rw & ((1u << 27) - 1), in_dim, X);
      }
      // layer-1 operand row (BF16, zero padded to K = 48)
#pragma unroll
      for (int k = 0; k < kK1; k += 2) {
        const float x0 = (k < kMaxIn && k < in_dim) ? X[k < kMaxIn ? k : 0] : 0.f;
        const float x1 = (k + 1 < kMaxIn && k + 1 < in_dim) ? X[k + 1 < kMaxIn ? k + 1 : 0] : 0.f;
        *reinterpret_cast<__nv_bfloat162*>(A1b + kmaj_off(tid, k, kK1)) = __floats2bfloat162_rn(x0, x1);
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
#pragma unroll
      for (int kk = 0; kk < kK1 / 16; ++kk)
        mma_bf16(tmem, make_desc(a1 + kk * 256, 128, (kK1 / 8) * 128), make_desc(b1s + kk * 256, 128, (kK1 / 8) * 128),
                 kIdesc1, kk > 0 ? 1u : 0u);
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase))) { timed_out = true; break; }
    phase ^= 1u;
    fence_after();
    if (row_thread) {
      float h[32];
      tmem_ld32(tmem + lane_base, h);
      // hidden layer: ReLU(D1 + b1) -> layer-2 operand row (BF16)
#pragma unroll
      for (int k = 0; k < kK2; k += 2) {
        const float h0 = fmaxf(h[k] + sm.b1[k], 0.f), h1 = fmaxf(h[k + 1] + sm.b1[k + 1], 0.f);
        *reinterpret_cast<__nv_bfloat162*>(A2b + kmaj_off(tid, k, kK2)) = __floats2bfloat162_rn(h0, h1);
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
#pragma unroll
      for (int kk = 0; kk < kK2 / 16; ++kk)
        mma_bf16(tmem + kD2Col, make_desc(a2 + kk * 256, 128, (kK2 / 8) * 128),
                 make_desc(b2s + kk * 256, 128, (kK2 / 8) * 128), kIdesc2, kk > 0 ? 1u : 0u);
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase))) { timed_out = true; break; }
    phase ^= 1u;
    fence_after();
    // epilogue: this thread's row and part of its Gaussians (column groups of two Gaussians)
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
    const int j_lo = epi_first(epart), j_hi = epart == 2 ? kNOff : epi_first(epart + 1);
#pragma unroll 1
    for (int grp = j_lo / 2; grp <= (j_hi - 1) / 2; ++grp) {
      float zc[32];
      tmem_ld32(tmem + lane_base + kD2Col + grp * kGroupCols, zc);
      if (valid) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int j = 2 * grp + u;
          if (j < j_lo || j >= j_hi) continue;
          float z[kPerGauss];
#pragma unroll
          for (int t = 0; t < kPerGauss; ++t) z[t] = zc[kPerGauss * u + t] + sm.b2p[grp * kGroupCols + kPerGauss * u + t];
          decode_gaussian(b, b.v[vi], z, l, xa, A.offsets + (a * kNOff + j) * 3, r * kNOff + j, rec, counts, keys, dec);
        }
      }
    }
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace pgs
