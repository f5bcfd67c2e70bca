// pa_noalloc.cu — pa_resample_counts_noalloc: the copy numbers, scan and parent
// map of one resampling, for callers that cannot allocate device memory.
//
// The block totals of the scan live in a file-scope __device__ array of fixed
// size instead of memory allocated per call.  Every GPU that loads libpa.so
// holds this array (32 KiB) until the process exits; all calls on a device share
// it, so calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it and must be serialised by the caller.  Each call
// writes every entry it later reads (the block totals, then their offsets, then
// the call's error mark), so nothing has to start at zero.
//
// Host code must not pass the array's name to a kernel: in host code it is a
// host-side stand-in, not a device address.  The device address is looked up
// with cudaGetSymbolAddress once per device, with that device current, on the
// first call made on it.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "../../include/pa.h"
#include "pa_device.cuh"
#include "pa_internal.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaSlotsPerBlock = 1024;  // four old slots per thread
constexpr int kNaMaxDevices = 64;

// [0, n_blocks): block totals, replaced by the scan with the blocks' offsets
// (64-bit: a block of 1024 slots may hold up to 2^41 copies); [n_blocks]: the
// call's error mark (nonzero when an input was invalid).  A block whose inputs
// are invalid writes -1 as its total.
__device__ __align__(256) long long g_na_scratch[PA_NOALLOC_MAX_BLOCKS + 1];

__device__ __forceinline__ long long warp_inclusive_scan_ll(long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive block scan of one 64-bit value per thread; sh holds 33 entries.
__device__ long long block_exclusive_scan_ll(long long v, long long* sh, long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long inc = warp_inclusive_scan_ll(v);
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const long long x = lane < nw ? sh[lane] : 0;
    const long long xi = warp_inclusive_scan_ll(x);
    if (lane < nw) sh[lane] = xi - x;
    if (lane == nw - 1) sh[32] = xi;
  }
  __syncthreads();
  const long long out = sh[warp] + inc - v;
  if (total) *total = sh[32];
  __syncthreads();
  return out;
}

// Copy numbers n_i = fl(k_i) + [r_i < thr(k_i)] of 1024 old slots per block; the
// block total goes to the static scratch.  A level outside [0, n_levels) or a
// floor entry outside [0, 2^31 - 2] is invalid: that slot's count is written as 0
// and the block's total as -1.
__global__ void __launch_bounds__(kNaThreads) k_na_counts(const int32_t* __restrict__ levels, int n_old,
                                                          const int32_t* __restrict__ fl,
                                                          const uint32_t* __restrict__ thr, int n_levels,
                                                          uint32_t k0, uint32_t k1, int t, int32_t* counts,
                                                          long long* scratch) {
  __shared__ long long red[kNaThreads / 32];
  const int i0 = blockIdx.x * kNaSlotsPerBlock + 4 * threadIdx.x;
  long long sum = 0;
  int bad = 0;
  if (i0 < n_old) {
    const uint4 r = pa::philox4x32_10(make_uint4((uint32_t)(i0 >> 2), 0u, 0u, (uint32_t)t), k0, k1);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + b;
      if (i < n_old) {
        const int k = levels[i];
        int n = 0;
        if (k < 0 || k >= n_levels) {
          bad = 1;
        } else {
          const int f = fl[k];
          if (f < 0 || f == INT_MAX)
            bad = 1;
          else
            n = f + (pa::word_of(r, b) < thr[k] ? 1 : 0);
        }
        counts[i] = n;
        sum += n;
      }
    }
  }
  bad = __syncthreads_or(bad);
  sum = pa::warp_sum(sum);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int w = 0; w < kNaThreads / 32; ++w) s += red[w];
    scratch[blockIdx.x] = bad ? -1 : s;
  }
}

// Exclusive scan of the block totals in the scratch (one block); the grand total
// is the new population size, or -1 when a block reported invalid input.
__global__ void k_na_scan(int n_blocks, long long* scratch, int64_t* n_new) {
  __shared__ long long sh[33];
  long long carry = 0;
  int bad = 0;
  for (int b0 = 0; b0 < n_blocks; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    const long long v = b < n_blocks ? scratch[b] : 0;
    bad |= __syncthreads_or(v < 0);
    long long tot;
    const long long ex = block_exclusive_scan_ll(v < 0 ? 0 : v, sh, &tot);
    if (b < n_blocks) scratch[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    scratch[n_blocks] = bad;
    *n_new = bad ? -1 : carry;
  }
}

// Parents of the new slots j < cap: slot offset_i + q (q < n_i) descends from old
// slot i.  Writes nothing when the call's inputs were invalid.
__global__ void __launch_bounds__(kNaThreads) k_na_scatter(const int32_t* __restrict__ counts, int n_old, int n_blocks,
                                                           const long long* __restrict__ scratch, int32_t* parents,
                                                           long long cap) {
  __shared__ long long sh[33];
  if (scratch[n_blocks] != 0) return;  // the same value for every thread of the grid
  const int i0 = blockIdx.x * kNaSlotsPerBlock + 4 * threadIdx.x;
  long long n[4] = {0, 0, 0, 0};
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (i0 + b < n_old) n[b] = counts[i0 + b];
  long long off = block_exclusive_scan_ll(n[0] + n[1] + n[2] + n[3], sh, nullptr) + scratch[blockIdx.x];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    for (long long j = off; j < off + n[b] && j < cap; ++j)
      if (j >= 0) parents[j] = i0 + b;
    off += n[b];
  }
}

std::mutex g_na_mutex;
long long* g_na_scratch_dev[kNaMaxDevices] = {};

// Device address of the scratch on the current device (looked up on first use).
int na_scratch(long long** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return PA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return PA_ERR_CUDA;
    g_na_scratch_dev[dev] = static_cast<long long*>(p);
  }
  *out = g_na_scratch_dev[dev];
  return PA_OK;
}

}  // namespace

extern "C" int pa_resample_counts_noalloc(const int32_t* levels, int64_t n_old, const int32_t* fl,
                                          const uint32_t* thr, int32_t n_levels, uint64_t run_seed, int32_t pop,
                                          int32_t t, int32_t* counts, int32_t* parents, int64_t parents_cap,
                                          int64_t* n_new, void* cuda_stream) {
  if (n_old < 0 || n_old > (int64_t)PA_NOALLOC_MAX_BLOCKS * kNaSlotsPerBlock) return PA_ERR_INVALID;
  if (!n_new || n_levels < 1 || parents_cap < 0 || pop < 0 || pop > 15 || t < 0 ||
      run_seed >= ((uint64_t)1 << 56))
    return PA_ERR_INVALID;
  if (n_old > 0 && (!levels || !fl || !thr || !counts)) return PA_ERR_INVALID;
  if (parents_cap > 0 && !parents) return PA_ERR_INVALID;
  long long* scratch = nullptr;
  int rc = na_scratch(&scratch);
  if (rc != PA_OK) return rc;
  const uint32_t k0 = (uint32_t)(run_seed & 0xffffffffu);
  const uint32_t k1 = (uint32_t)(run_seed >> 32) | ((uint32_t)pa::kResample << 28) | ((uint32_t)pop << 24);
  const int n_blocks = (int)((n_old + kNaSlotsPerBlock - 1) / kNaSlotsPerBlock);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (n_blocks > 0)
    k_na_counts<<<n_blocks, kNaThreads, 0, s>>>(levels, (int)n_old, fl, thr, n_levels, k0, k1, t, counts, scratch);
  k_na_scan<<<1, 1024, 0, s>>>(n_blocks, scratch, n_new);
  if (n_blocks > 0)
    k_na_scatter<<<n_blocks, kNaThreads, 0, s>>>(counts, (int)n_old, n_blocks, scratch, parents,
                                                 (long long)parents_cap);
  return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}
