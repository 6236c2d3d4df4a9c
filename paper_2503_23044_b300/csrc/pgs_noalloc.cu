// Radix sort of key/value pairs that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a sort:
// code running inside an allocator or a memory-pool callback, plug-ins whose
// host framework owns all device memory and forbids side allocations, or
// real-time paths that must not risk an allocation failure or the implicit
// device synchronisation a fresh cudaMalloc may cause.  pgs_sort_pairs needs
// a caller-provided scratch buffer plus two ping-pong arrays; this variant
// keeps all of that in one fixed-size array that lives in the library's own
// device image (a file-scope __device__ array), so the caller passes only the
// keys and values.
//
// The array holds the device copy of n, the digit histograms, the look-back
// status words and the ping-pong keys/values for at most kNoAllocMaxN pairs,
// about 9.4 MB; every GPU that loads the library keeps it until the process
// exits.  Host code cannot use the array's name as a device address, so every
// call looks the address up with cudaGetSymbolAddress on the current device
// (a cheap host call; nothing is cached, so the address is never stale after
// a context is torn down and re-created).
//
// Under CUDA's lazy module loading the first call on a device can load this
// file's device code, which is when the array is reserved, and it runs the
// sort's one-time launch set-up (carveout and occupancy query).  The
// allocation-free guarantee therefore holds from the second call on: warm up
// each device with one call (any n >= 1) first, outside any stream capture.
#include <cstdio>

#include "pgs_internal.cuh"
#include "pgs_kernels.cuh"

namespace {

constexpr long long kNoAllocMaxN = 1ll << 20;
constexpr size_t kNoAllocHeader = 256;   // n (int64) + error word, padded
constexpr size_t kNoAllocSortBytes = pgs::sort_scratch_bytes_for(kNoAllocMaxN);
constexpr size_t kNoAllocPing = (size_t)kNoAllocMaxN * 4;
constexpr size_t kNoAllocBytes =
    kNoAllocHeader + ((kNoAllocSortBytes + 255) / 256) * 256 + 2 * kNoAllocPing;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void k_noalloc_setup(long long* d_n, long long n, uint32_t* err) {
  *d_n = n;
  *err = 0u;
}

thread_local char g_msg[256];

pgs_status fail_na(pgs_status s) {
  pgs::set_last_error(g_msg);
  return s;
}

}  // namespace

extern "C" {

pgs_status pgs_sort_pairs_noalloc(uint32_t* d_keys, uint32_t* d_vals, int64_t n, int bit_lo, int bit_hi,
                                  uint32_t* d_err, cudaStream_t stream) {
  g_msg[0] = 0;
  if (n < 0 || n > kNoAllocMaxN) {
    snprintf(g_msg, sizeof(g_msg), "pgs_sort_pairs_noalloc: n = %lld is outside [0, %lld], the size of its fixed scratch",
             (long long)n, kNoAllocMaxN);
    return fail_na(PGS_ERR_INVALID_ARG);
  }
  if (n > 0 && (!d_keys || !d_vals)) {
    snprintf(g_msg, sizeof(g_msg), "pgs_sort_pairs_noalloc: null keys or values");
    return fail_na(PGS_ERR_INVALID_ARG);
  }
  if (bit_lo < 0 || bit_hi > 32 || bit_lo >= bit_hi) {
    snprintf(g_msg, sizeof(g_msg), "pgs_sort_pairs_noalloc: bit range [%d, %d)", bit_lo, bit_hi);
    return fail_na(PGS_ERR_INVALID_ARG);
  }
  // set-up on the current device: the device address of the array (looked up on every call)
  void* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
  if (e != cudaSuccess || !base) {
    snprintf(g_msg, sizeof(g_msg), "pgs_sort_pairs_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    return fail_na(PGS_ERR_CUDA);
  }
  if (n == 0) return PGS_OK;
  unsigned char* b = static_cast<unsigned char*>(base);
  long long* d_n = reinterpret_cast<long long*>(b);
  uint32_t* own_err = reinterpret_cast<uint32_t*>(b + 8);
  void* sort_base = b + kNoAllocHeader;
  uint32_t* alt_k = reinterpret_cast<uint32_t*>(b + kNoAllocHeader + ((kNoAllocSortBytes + 255) / 256) * 256);
  uint32_t* alt_v = alt_k + kNoAllocMaxN;
  pgs::SortScratch ss = pgs::sort_scratch_layout(sort_base, kNoAllocMaxN);
  // n and the error word start each call fresh (the array keeps the last call's contents)
  k_noalloc_setup<<<1, 1, 0, stream>>>(d_n, (long long)n, own_err);
  const int ns = pgs::device_sm_count();
  e = pgs::launch_sort_pairs(d_keys, d_vals, alt_k, alt_v, d_n, kNoAllocMaxN, bit_lo, bit_hi, ss,
                             d_err ? d_err : own_err, 1u << 20, pgs::kNoHoldTile, ns, stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof(g_msg), "pgs_sort_pairs_noalloc: launch: %s", cudaGetErrorString(e));
    return fail_na(PGS_ERR_CUDA);
  }
  return PGS_OK;
}

}  // extern "C"
