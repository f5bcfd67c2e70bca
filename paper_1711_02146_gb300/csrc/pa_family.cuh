// pa_family.cuh — accumulation of the family statistics of a step (§III.A):
// the sum of eta^2 over families (rho_t), the number of families, and the sum of
// nu ln nu with nu = eta / R~ (the family entropy S_f = -sum, and rho_s).
//
// The blocks that find families add eta^2 and the family count with integer
// atomics, and count each family in the step's size histogram fhist; the first
// family of a size also appends the size to the list fsizes.  The last block to
// finish then adds m(eta) nu ln nu once per listed size (a population of R~ has at
// most sqrt(2 R~) distinct family sizes, so few FP64 logarithms), clears the
// histogram entries and the counters for the next step, and stores the sum.
//
// nu ln nu is summed as a 128-bit fixed-point number in units of 2^-100: with
// R~ < 2^31, a nonzero |m nu ln nu| exceeds 2^-27, so its last bit is 2^-79 or
// coarser and the scaled value is an integer; the conversion is exact, and the
// sum is exact and independent of its order (and of the launch shape).  The
// host rounds it to double once.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pa_internal.h"

namespace pa {

struct FamilyAcc {
  unsigned long long s2 = 0, nf = 0;
  __device__ __forceinline__ void add(int eta) {
    s2 += (unsigned long long)eta * (unsigned long long)eta;
    nf += 1;
  }
};

// The lanes of thread tid's warp in a CTA of nthreads threads.
__device__ __forceinline__ unsigned warp_lanes(int tid, int nthreads) {
  const int first = tid & ~31;
  return nthreads - first >= 32 ? 0xffffffffu : (1u << (nthreads - first)) - 1u;
}

// Counts one family of size eta (0: none) in the step's size histogram; all lanes
// in `mask` call it together.  Lanes with the same size add with one atomic, and
// the lane that takes a size from zero appends it to the size list.
__device__ __forceinline__ void family_size(const PopDev& P, int eta, unsigned mask) {
  const unsigned peers = __match_any_sync(mask, eta);
  if (eta > 0 && (int)(threadIdx.x & 31u) == __ffs(peers) - 1) {
    if (atomicAdd(&P.fhist[eta], __popc(peers)) == 0) P.fsizes[atomicAdd(&P.fcount[0], 1)] = eta;
  }
}

// Adds a CTA's sum of eta^2 and family count to the step record (each warp
// reduces; lane 0 of every warp adds with global atomics).
__device__ __forceinline__ void family_flush(FamilyAcc f, unsigned mask, StepRec* rec) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long s2o = __shfl_xor_sync(mask, f.s2, o), nfo = __shfl_xor_sync(mask, f.nf, o);
    if (mask >> ((threadIdx.x & 31u) ^ (unsigned)o) & 1u) {  // a lane outside the mask contributes nothing
      f.s2 += s2o;
      f.nf += nfo;
    }
  }
  if ((threadIdx.x & 31u) == 0 && f.nf) {
    atomicAdd(&rec->sum_eta2, f.s2);
    atomicAdd(&rec->n_families, f.nf);
  }
}

// m nu ln nu (nu = eta / R~) in units of 2^-100 as (hi, lo): value = hi 2^64 + lo.
__device__ __forceinline__ void entropy_term(int m, int eta, int R_new, long long& hi, unsigned long long& lo) {
  const double nu = __ddiv_rn((double)eta, (double)R_new);
  const double v = __dmul_rn(__dmul_rn((double)m, __dmul_rn(nu, log(nu))), 0x1p100);  // an integer, <= 0
  const double h = floor(__dmul_rn(v, 0x1p-64));
  hi = (long long)h;
  lo = (unsigned long long)__dsub_rn(v, __dmul_rn(h, 0x1p64));
}

__device__ __forceinline__ void add128(long long& hi, unsigned long long& lo, long long h, unsigned long long l) {
  const unsigned long long s = lo + l;
  hi += h + (s < lo ? 1 : 0);
  lo = s;
}

// Called by every thread of each of the `participants` CTAs that found families of
// this step, after their family_size and family_flush calls.  The last of them
// adds the entropy terms of the listed sizes into rec (an exact 128-bit sum),
// clears the histogram entries it read and the counters.  sh: 64 words of shared
// memory.
__device__ __forceinline__ void family_entropy_last(const PopDev& P, StepRec* rec, int R_new, int participants,
                                                    int tid, int nthreads, long long* sh) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&P.fcount[1], 1) == participants - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int K = __ldcg(&P.fcount[0]);
  long long hi = 0;
  unsigned long long lo = 0;
  for (int k = tid; k < K; k += nthreads) {
    const int eta = __ldcg(&P.fsizes[k]);
    const int m = __ldcg(&P.fhist[eta]);
    long long h;
    unsigned long long l;
    entropy_term(m, eta, R_new, h, l);
    add128(hi, lo, h, l);
    P.fhist[eta] = 0;
  }
  const unsigned mask = warp_lanes(tid, nthreads);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ho = __shfl_xor_sync(mask, hi, o);
    const unsigned long long lw = __shfl_xor_sync(mask, lo, o);
    if (mask >> ((threadIdx.x & 31u) ^ (unsigned)o) & 1u) add128(hi, lo, ho, lw);
  }
  const int nw = (nthreads + 31) / 32;
  if ((tid & 31) == 0) {
    sh[2 * (tid >> 5)] = hi;
    sh[2 * (tid >> 5) + 1] = (long long)lo;
  }
  __syncthreads();
  if (tid == 0) {
    long long H = 0;
    unsigned long long Lo = 0;
    for (int w = 0; w < nw; ++w) add128(H, Lo, sh[2 * w], (unsigned long long)sh[2 * w + 1]);
    rec->nll_hi = H;
    rec->nll_lo = Lo;
    P.fcount[0] = 0;
    P.fcount[1] = 0;
  }
}

// First slot at or after `from` whose label differs from l (R_new if none): the
// labels ascend along the slots, so probe from, from + 1, + 3, + 7, ... and then
// bisect the last gap.  At most about 2 log2(R_new) loads.
__device__ __forceinline__ int run_end(const int32_t* __restrict__ lab, int l, int from, int R_new) {
  if (from >= R_new) return R_new;
  if (lab[from] != l) return from;
  int lo = from, step = 1, hi;  // lab[lo] == l
  for (;;) {
    const long long nxt = (long long)lo + step;
    if (nxt >= R_new || lab[nxt] != l) {
      hi = nxt >= R_new ? R_new : (int)nxt;
      break;
    }
    lo = (int)nxt;
    step <<= 1;
  }
  while (hi - lo > 1) {  // lab[lo] == l; hi is R_new or lab[hi] != l
    const int mid = lo + ((hi - lo) >> 1);
    if (lab[mid] == l)
      lo = mid;
    else
      hi = mid;
  }
  return hi;
}

}  // namespace pa
