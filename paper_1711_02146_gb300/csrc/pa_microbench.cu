// pa_microbench.cu — integer issue-rate probes (include/pa_bench.h).
// Each thread runs 8 independent chains so that issue rate, not latency, limits.
#include <cuda_runtime.h>

#include "../../include/pa.h"
#include "../../include/pa_bench.h"
#include "pa_device.cuh"

namespace {

__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t add_u32(uint32_t a, uint32_t b) {
  uint32_t d;
  asm volatile("add.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t mulwide_fold(uint32_t a, uint32_t m) {
  uint64_t p;
  asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(m));
  uint32_t lo = (uint32_t)p, hi = (uint32_t)(p >> 32);
  return lop3_xor(lo, hi, a);
}

__device__ __forceinline__ uint32_t mulwide_add(uint32_t a, uint32_t m) {
  uint64_t p;
  asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(m));
  return add_u32((uint32_t)p, (uint32_t)(p >> 32));
}

template <int KIND>
__global__ void k_probe(int64_t iters, uint32_t seed, uint32_t* out) {
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = gid * 2654435761u + seed + (uint32_t)i * 40503u;
  const uint32_t b = seed ^ 0x9E3779B9u, c = seed + 0x7F4A7C15u;
  if constexpr (KIND == PA_BENCH_PHILOX || KIND == PA_BENCH_PHILOX_LOP3) {
    uint32_t acc = 0;
    for (int64_t it = 0; it < iters; ++it) {
      const uint4 r = pa::philox4x32_10(make_uint4(gid, (uint32_t)it, x[0], seed), b, c);
      acc ^= r.x ^ r.y ^ r.z ^ r.w;
      if (KIND == PA_BENCH_PHILOX_LOP3) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = lop3_xor(lop3_xor(x[i], b, c), c, b);  // independent of the block
      }
    }
    uint32_t fold = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) fold ^= x[i];
    out[gid] = acc ^ (KIND == PA_BENCH_PHILOX_LOP3 ? fold : 0u);
  } else {
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (KIND == PA_BENCH_LOP3) x[i] = lop3_xor(x[i], b, c);
        if (KIND == PA_BENCH_IADD) x[i] = add_u32(x[i], b);
        if (KIND == PA_BENCH_IMAD) x[i] = mad_lo(x[i], b, c);
        if (KIND == PA_BENCH_MULWIDE) x[i] = mulwide_fold(x[i], b);
        if (KIND == PA_BENCH_MULWIDE_ADD) x[i] = mulwide_add(x[i], b);
        if (KIND == PA_BENCH_LOP3_IADD) x[i] = add_u32(lop3_xor(x[i], b, c), c);
      }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    out[gid] = acc;
  }
}

template <int KIND>
int run_probe(int64_t iters, int blocks, int threads, double* ms) {
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, sizeof(uint32_t) * (size_t)blocks * threads) != cudaSuccess) return PA_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_probe<KIND><<<blocks, threads>>>(iters / 8 + 1, 1u, out);  // warm-up
  cudaEventRecord(e0);
  k_probe<KIND><<<blocks, threads>>>(iters, 12345u, out);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float f = 0.f;
  cudaEventElapsedTime(&f, e0, e1);
  *ms = f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

}  // namespace

extern "C" int pa_bench_int_throughput(int kind, int64_t iters, int blocks, int threads, double* ms, double* ops) {
  if (!ms || !ops || iters < 1 || blocks < 1 || threads < 32 || threads > 1024) return PA_ERR_INVALID;
  const double n = (double)blocks * threads * (double)iters;
  switch (kind) {
    case PA_BENCH_LOP3: *ops = 8 * n; return run_probe<PA_BENCH_LOP3>(iters, blocks, threads, ms);
    case PA_BENCH_IADD: *ops = 8 * n; return run_probe<PA_BENCH_IADD>(iters, blocks, threads, ms);
    case PA_BENCH_IMAD: *ops = 8 * n; return run_probe<PA_BENCH_IMAD>(iters, blocks, threads, ms);
    case PA_BENCH_MULWIDE: *ops = 16 * n; return run_probe<PA_BENCH_MULWIDE>(iters, blocks, threads, ms);
    case PA_BENCH_PHILOX: *ops = 4 * n; return run_probe<PA_BENCH_PHILOX>(iters, blocks, threads, ms);
    case PA_BENCH_MULWIDE_ADD: *ops = 16 * n; return run_probe<PA_BENCH_MULWIDE_ADD>(iters, blocks, threads, ms);
    case PA_BENCH_LOP3_IADD: *ops = 16 * n; return run_probe<PA_BENCH_LOP3_IADD>(iters, blocks, threads, ms);
    case PA_BENCH_PHILOX_LOP3: *ops = 4 * n; return run_probe<PA_BENCH_PHILOX_LOP3>(iters, blocks, threads, ms);
    default: return PA_ERR_INVALID;
  }
}
