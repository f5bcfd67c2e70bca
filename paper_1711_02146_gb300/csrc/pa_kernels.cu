// pa_kernels.cu — initialisation, reweighting, resampling, family and overlap
// kernels of the population annealing step (Amey & Machta, §II, §III.A).
//
// Spin storage: int8 +1 (0x01) / -1 (0xFF), site-major: row n holds all slots of
// site n contiguously (pitch bytes), so one 32-bit word carries four replicas
// of one site.  For two spins a, b of that encoding a ^ b is 0x00 when equal and
// 0xFE when different; XOR with a coupling mask (0xFE for J = -1, else 0) gives
// 0xFE exactly for an unsatisfied bond, and bit 1 of each byte counts it.
#include <cuda_runtime.h>

#include "pa_device.cuh"
#include "pa_family.cuh"
#include "pa_internal.h"

namespace pa {

struct PopArgs {
  PopDev p[2];
};

static PopArgs pack(const PopDev* pops, int n_pop) {
  PopArgs a;
  for (int i = 0; i < n_pop && i < 2; ++i) a.p[i] = pops[i];
  return a;
}

constexpr uint32_t kBit1 = 0x02020202u;
constexpr int kScatterOwn = 16;  // copies a thread writes alone; larger families are written by the warp

// ---------------------------------------------------------------- init (a0)

// Couplings J(n, d) = +1 if bit 0 of Philox word d at counter (n, 0, 0, 0) is 0.
// jtab[4n + d] is the XOR mask of the forward bond (n, d).
__global__ void k_init_couplings(int N, uint32_t k0, uint32_t k1, int8_t* J, uint32_t* jtab) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)n, 0u, 0u, 0u), k0, k1);
  const uint32_t w[3] = {r.x, r.y, r.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const bool neg = (w[d] & 1u) != 0;
    J[3 * n + d] = neg ? (int8_t)-1 : (int8_t)1;
    jtab[4 * n + d] = neg ? 0xFEFEFEFEu : 0u;
  }
  jtab[4 * n + 3] = 0u;
}

// Initial spins: slot j at site n is +1 if bit 0 of word (j & 3) of Philox at
// counter (n, 0, j >> 2, 0) is 0, else -1, j the global slot (slot_base + local
// slot); slots past the initial population are padded with +1.
__global__ void k_init_population(RunGeom g, PopArgs a, int cur) {
  const int pop = blockIdx.y;
  const PopDev& P = a.p[pop];
  const int64_t words = g.pitch / 4;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= words * g.N) return;
  const int n = (int)(gid / words);
  const uint32_t wi = (uint32_t)(gid % words);
  const uint32_t gw = (uint32_t)(g.slot_base / 4) + wi;  // global word (slot_base is a multiple of 4)
  const uint4 r = philox4x32_10(make_uint4((uint32_t)n, 0u, gw, 0u), P.key_init[0], P.key_init[1]);
  uint32_t out = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int64_t j = 4 * (int64_t)wi + b;
    const uint32_t byte = (j < g.n_init && (word_of(r, b) & 1u)) ? 0xFFu : 0x01u;
    out |= byte << (8 * b);
  }
  reinterpret_cast<uint32_t*>(P.spins[cur] + (size_t)n * g.pitch)[wi] = out;
  if (n == 0) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t j = 4 * (int64_t)wi + b;
      if (j < g.n_init) P.labels[cur][j] = (int32_t)(g.slot_base + j);
    }
  }
  if (n == 0 && wi == 0) P.rec[0].R_tilde = g.n_init;
}

// Energy level (unsatisfied bonds) of every slot from scratch, and the level
// histogram of step t.  One thread per word (four replicas).
__global__ void k_levels_and_hist(RunGeom g, PopArgs a, int cur, const uint32_t* __restrict__ jtab, int t) {
  const int pop = blockIdx.y;
  const PopDev& P = a.p[pop];
  const int R = P.rec[t].R_tilde;
  const int wi = blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * wi >= R) return;
  const int L = g.L;
  const uint32_t* S = reinterpret_cast<const uint32_t*>(P.spins[cur]);
  const int64_t pw = g.pitch / 4;
  int cnt[4] = {0, 0, 0, 0};
  uint32_t acc = 0;
  int since = 0;
  for (int n = 0; n < g.N; ++n) {
    const int x = n % L, y = (n / L) % L, z = n / (L * L);
    const int nx = (x + 1 == L ? 0 : x + 1) + L * (y + L * z);
    const int ny = x + L * ((y + 1 == L ? 0 : y + 1) + L * z);
    const int nz = x + L * (y + L * (z + 1 == L ? 0 : z + 1));
    const uint32_t s = S[n * pw + wi];
    acc += ((s ^ S[nx * pw + wi] ^ jtab[4 * n + 0]) & kBit1) + ((s ^ S[ny * pw + wi] ^ jtab[4 * n + 1]) & kBit1) +
           ((s ^ S[nz * pw + wi] ^ jtab[4 * n + 2]) & kBit1);
    if (++since == 40) {
#pragma unroll
      for (int b = 0; b < 4; ++b) cnt[b] += (acc >> (8 * b)) & 0xFFu;
      acc = 0;
      since = 0;
    }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) cnt[b] += (acc >> (8 * b)) & 0xFFu;
  uint32_t* hist = P.hist + (size_t)t * g.n_levels;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = 4 * wi + b;
    if (j < R) {
      const int k = cnt[b] >> 1;
      P.levels[j] = k;
      atomicAdd(&hist[k], 1u);
    }
  }
}

// ---------------------------------------------------------------- reweight (a4)

// One block per population.  From the level histogram c of step t-1 and the
// weights w[j] = exp(-dbeta 2j) (computed on the host in FP64):
//   S' = sum_{k >= kmin} c(k) w[k - kmin]         (ascending k, separate mul/add)
//   tau_k = R w[k - kmin] / S'  ->  fl_k = floor(tau_k), thr_k = 2^32 (tau_k - fl_k)
//   eps = (1/R) sum_k c(k) (1 - tau_k)_+          (Eq. eq_num_elim; fixed tree order)
// Empty levels add exact zeros to S', so they are skipped there.
// One block per population; lst_sh (n_levels entries) holds the occupied levels,
// ascending, when list_in_smem.
__device__ __forceinline__ void reweight_pop(const RunGeom& g, const PopDev& P, const double* __restrict__ w, int t,
                                             int* lst_sh, int list_in_smem) {
  __shared__ int scratch[33];
  __shared__ double S_sh;
  if (threadIdx.x == 0) *P.ticket = 0;  // the tile ticket of this step's single-pass resampling
  // the list lives in shared memory when it fits; otherwise in the floor table,
  // which is only written (below) after the list has been read
  int* lst = list_in_smem ? lst_sh : P.fl;
  const uint32_t* c = P.hist + (size_t)(t - 1) * g.n_levels;
  int base = 0;
  for (int k0 = 0; k0 < g.n_levels; k0 += blockDim.x) {
    const int k = k0 + threadIdx.x;
    const int f = (k < g.n_levels && c[k] > 0u) ? 1 : 0;
    int tot;
    const int pos = block_exclusive_scan(f, scratch, &tot);
    if (f) lst[base + pos] = k;
    base += tot;
  }
  __syncthreads();
  const int nnz = base;
  if (nnz == 0) return;  // cannot happen: the population is never empty here
  const int kmin = lst[0];
  // S' = the sum over occupied levels, ascending, of c(k) w(k - kmin): every thread
  // forms products, 1024 at a time, into shared memory, and one thread adds them in
  // level order (the operations and their order of a single thread)
  __shared__ double eps_sh[1024];  // the products here, the culling sums below
  double acc = 0.0;
  for (int base = 0; base < nnz; base += blockDim.x) {
    const int i = base + threadIdx.x;
    if (i < nnz) {
      const int k = lst[i];
      eps_sh[threadIdx.x] = __dmul_rn((double)c[k], w[k - kmin]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int m = min(nnz - base, (int)blockDim.x);
      for (int j = 0; j < m; ++j) acc = __dadd_rn(acc, eps_sh[j]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) S_sh = acc;
  __syncthreads();
  const double S = S_sh;
  const double Rd = (double)g.R;
  double eps_part = 0.0;  // this thread's levels, ascending
  for (int k = threadIdx.x; k < g.n_levels; k += blockDim.x) {
    int f = 0;
    uint32_t th = 0u;
    if (k >= kmin) {
      const double tau = __ddiv_rn(__dmul_rn(Rd, w[k - kmin]), S);
      const double fl = floor(tau);
      f = (int)fl;
      th = (uint32_t)__dmul_rn(__dsub_rn(tau, fl), 4294967296.0);
      if (tau < 1.0 && c[k] > 0u) eps_part = __dadd_rn(eps_part, __dmul_rn((double)c[k], __dsub_rn(1.0, tau)));
    }
    P.fl[k] = f;
    P.thr[k] = th;
  }
  // expected culling fraction (Eq. eq_num_elim / R): fixed tree over the threads
  eps_sh[threadIdx.x] = eps_part;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) eps_sh[threadIdx.x] = __dadd_rn(eps_sh[threadIdx.x], eps_sh[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    StepRec& r = P.rec[t];
    r.S_prime = S;
    r.eps_expected = __ddiv_rn(eps_sh[0], Rd);
    r.kmin_prev = kmin;
    r.R_prev = P.rec[t - 1].R_tilde;
  }
}

__global__ void k_reweight(RunGeom g, PopArgs a, const double* __restrict__ w, int t, int list_in_smem) {
  extern __shared__ int lst_sh[];
  reweight_pop(g, a.p[blockIdx.x], w, t, lst_sh, list_in_smem);
}

// Every unit of a batch, one block each; the step record of the round's step is
// cleared here (a lone run clears it with a memset before this kernel).
__global__ void k_group_reweight(const GroupUnit* __restrict__ units, const int32_t* __restrict__ round) {
  extern __shared__ int lst_sh[];
  const GroupUnit& u = units[blockIdx.x];
  const int t = u.t0 + 1 + *round;
  if (t > u.last_t) return;
  if (threadIdx.x == 0) u.P.rec[t] = StepRec{};
  reweight_pop(u.g, u.P, u.steps[t].w, t, lst_sh, 1);
}

// ---------------------------------------------------------------- resampling (a5, a6)

// Exclusive scan of per-block copy totals (one block per population; the
// Gaussian model's resampling); the grand total is the new population size R~_t.  A total above R_cap sets the capacity
// flag and is clamped so that no later kernel writes out of bounds.
__global__ void k_scan_blocks(RunGeom g, PopArgs a, int t, int32_t* status) {
  __shared__ int scratch[33];
  const PopDev& P = a.p[blockIdx.x];
  long long carry = 0;
  for (int b0 = 0; b0 < g.n_count_blocks; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    const int v = b < g.n_count_blocks ? P.blocksums[b] : 0;
    int tot;
    const int ex = block_exclusive_scan(v, scratch, &tot);
    const long long off = carry + ex;
    if (b < g.n_count_blocks) P.blocksums[b] = off > 0x7fffffffLL ? 0x7fffffff : (int)off;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    int R_new = carry > g.R_cap ? g.R_cap : (int)carry;
    if (carry > g.R_cap) atomicOr(status, kFlagCapacity);
    if (carry == 0) atomicOr(status, kFlagExtinct);
    P.rec[t].R_tilde = R_new;
  }
}

// New population: slot offsets[i] + q (q < n_i) takes old slot i as parent and
// inherits its family label, so labels stay sorted along the slots.
__global__ void __launch_bounds__(kCountThreads) k_scatter(RunGeom g, PopArgs a, int cur, int t) {
  __shared__ int scratch[33];
  const PopDev& P = a.p[blockIdx.y];
  const int R_old = P.rec[t - 1].R_tilde;
  const int i0 = blockIdx.x * kSlotsPerCountBlock + 4 * threadIdx.x;
  int n[4] = {0, 0, 0, 0};
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (i0 + b < R_old) n[b] = P.counts[i0 + b];
  const int local = n[0] + n[1] + n[2] + n[3];
  long long off = (long long)block_exclusive_scan(local, scratch, nullptr) + P.blocksums[blockIdx.x];
  const int32_t* lab_old = P.labels[cur];
  int32_t* lab_new = P.labels[1 - cur];
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int i = i0 + b;
    // a slot with few copies writes them itself; the copies of a large family are
    // written by the whole warp, one such slot at a time
    const bool big = n[b] > kScatterOwn;
    if (!big)
      for (int q = 0; q < n[b]; ++q) {
        const long long j = off + q;
        if (j < g.R_cap) {
          P.parents[j] = i;
          lab_new[j] = lab_old[i];
        }
      }
    unsigned int pending = __ballot_sync(0xffffffffu, big);
    while (pending) {
      const int src = __ffs(pending) - 1;
      pending &= pending - 1;
      const long long o = __shfl_sync(0xffffffffu, off, src);
      const int cnt = __shfl_sync(0xffffffffu, n[b], src);
      const int ii = __shfl_sync(0xffffffffu, i, src);
      const int32_t lab = lab_old[ii];
      for (int q = lane; q < cnt; q += 32) {
        const long long j = o + q;
        if (j < g.R_cap) {
          P.parents[j] = ii;
          lab_new[j] = lab;
        }
      }
    }
    off += n[b];
  }
}

// Single-pass resampling of the +-1 model (§II): copy numbers n_i = fl(k_i) +
// [r_i < thr(k_i)], r_i = word (i & 3) of Philox at counter (i >> 2, 0, 0, t) —
// the nearest-integer rule — their running offsets, and the new population's
// parents and labels (new slot offset_i + q, q < n_i, takes old slot i as parent
// and inherits its label, so labels stay sorted along the slots) in one launch.
// Tiles of kResampleTile old slots are numbered in the order blocks start (a ticket), so a
// block only ever waits on tiles whose blocks are already running or done.  Each
// block publishes its copy total, then walks back over its predecessors' entries
// (a total, or a total including everything before it), kCountThreads at a time,
// until it has its offset, and publishes that inclusive prefix.  Entries carry the step in their upper
// word (2t + 1: total, 2t + 2: inclusive), so older steps' entries read as not
// ready.  A wait gives up after spin_limit polls (kLookbackSpins unless a test
// lowers it) and sets the timeout flag.  A test may also name a tile whose block
// publishes neither its total nor its prefix (withheld >= 0), so that the waits of
// the blocks after it run out; -1 in normal runs.
constexpr int kResampleSlots = 4;  // old slots per thread (4096-slot tiles measured slower)
constexpr int kResampleTile = kResampleSlots * kCountThreads;  // old slots per tile

__device__ __forceinline__ unsigned long long poll_tile(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

static_assert(kResampleTile == kResampleSlotsPerBlock, "resampling blocks of a batch are counted by the host");

__device__ __forceinline__ void resample_pop(const RunGeom& g, const PopDev& P, int cur, int t, int32_t* status,
                                             int spin_limit, int withheld) {
  __shared__ int scratch[33];
  __shared__ int tile_sh;
  __shared__ long long base_sh;
  __shared__ unsigned incl_sh[kCountThreads / 32];
  __shared__ long long sum_sh[kCountThreads / 32];
  if (threadIdx.x == 0) tile_sh = atomicAdd(P.ticket, 1);
  __syncthreads();
  const int tile = tile_sh;
  const int R_old = P.rec[t - 1].R_tilde;
  // chunk m (m < kResampleSlots / 4) of the tile: slots base + 1024 m + 4 threadIdx.x + b, b < 4
  constexpr int kChunks = kResampleSlots / 4, kChunkSlots = 4 * kCountThreads;
  const int base = tile * kResampleTile;
  int n[kResampleSlots];
  int cul = 0, ex[kChunks], chunk_base[kChunks], total = 0;
#pragma unroll
  for (int m = 0; m < kChunks; ++m) {
    const int j0 = base + m * kChunkSlots + 4 * threadIdx.x;
    int local = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) n[4 * m + b] = 0;
    if (j0 < R_old) {  // the uniform of old slot i is addressed by its global slot slot_base + i
      const uint4 r = philox4x32_10(make_uint4((uint32_t)((g.slot_base + j0) >> 2), 0u, 0u, (uint32_t)t),
                                    P.key_res[0], P.key_res[1]);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = j0 + b;
        if (i < R_old) {
          const int k = P.levels[i];
          const int c = P.fl[k] + (word_of(r, b) < P.thr[k] ? 1 : 0);
          n[4 * m + b] = c;
          P.counts[i] = c;
          cul += (c == 0);
          local += c;
        }
      }
    }
    int tot;
    ex[m] = block_exclusive_scan(local, scratch, &tot);
    chunk_base[m] = total;
    total += tot;
  }
  cul = warp_sum(cul);
  if ((threadIdx.x & 31) == 0 && cul) atomicAdd(&P.rec[t].culled, cul);
  // Publish the total, then look back kCountThreads tiles at a time with the whole
  // block (thread x reads the entry of tile hi - x): the window's nearest inclusive
  // entry ends the walk, and only the entries nearer than it must be ready.  Every
  // decision is block-wide (__syncthreads_or, shared words), so all threads leave
  // the loops together.
  const uint32_t ep_total = 2u * (uint32_t)t + 1u, ep_incl = ep_total + 1u;
  if (threadIdx.x == 0 && tile > 0 && tile != withheld)
    atomicExch(&P.tiles[tile], ((unsigned long long)ep_total << 32) | (unsigned)total);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kWarps = kCountThreads / 32;
  long long prefix = 0;
  bool ok = true;
  for (int hi = tile - 1; hi >= 0; hi -= kCountThreads) {
    const int q = hi - (int)threadIdx.x;  // tiles before 0 read as an inclusive 0
    unsigned long long v = q >= 0 ? poll_tile(&P.tiles[q]) : ((unsigned long long)ep_incl << 32);
    int first = kCountThreads;  // nearest inclusive entry of the window (kCountThreads: none)
    for (int spins = 0;; ++spins) {
      const unsigned incl = __ballot_sync(0xffffffffu, (uint32_t)(v >> 32) == ep_incl);
      if (lane == 0) incl_sh[warp] = incl;
      __syncthreads();
      first = kCountThreads;
      for (int w = kWarps - 1; w >= 0; --w)
        if (incl_sh[w]) first = 32 * w + __ffs(incl_sh[w]) - 1;
      const bool waiting = (uint32_t)(v >> 32) < ep_total && (int)threadIdx.x < first;
      if (!__syncthreads_or(waiting)) break;  // also orders the reads of incl_sh before its next write
      if (spins >= spin_limit) {
        ok = false;
        break;
      }
      if (waiting) {
        __nanosleep(32);
        v = poll_tile(&P.tiles[q]);
      }
    }
    if (!ok) break;
    long long c = (int)threadIdx.x <= first ? (long long)(uint32_t)v : 0;
    c = warp_sum(c);
    if (lane == 0) sum_sh[warp] = c;
    __syncthreads();
    for (int w = 0; w < kWarps; ++w) prefix += sum_sh[w];
    __syncthreads();  // sum_sh is read before the next window writes it
    if (first < kCountThreads) break;
  }
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(status, kFlagTimeout);
    const long long inc = prefix + total;
    if (tile != withheld)
      atomicExch(&P.tiles[tile], ((unsigned long long)ep_incl << 32) | (unsigned)(inc > 0x7fffffffLL ? 0x7fffffffLL : inc));
    base_sh = prefix;
    // the tile holding the last old slot (tile 0 for an empty population) records R~
    if (tile == (R_old > 0 ? (R_old - 1) / kResampleTile : 0)) {
      P.rec[t].R_tilde = inc > g.R_cap ? g.R_cap : (int)inc;
      if (inc > g.R_cap) atomicOr(status, kFlagCapacity);
      if (inc == 0) atomicOr(status, kFlagExtinct);
    }
  }
  __syncthreads();
  const int32_t* lab_old = P.labels[cur];
  int32_t* lab_new = P.labels[1 - cur];
#pragma unroll
  for (int m = 0; m < kChunks; ++m) {
    long long off = base_sh + chunk_base[m] + ex[m];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = base + m * kChunkSlots + 4 * threadIdx.x + b;
      const int nb = n[4 * m + b];
      const bool big = nb > kScatterOwn;  // a large family is written by the whole warp
      if (!big)
        for (int q = 0; q < nb; ++q) {
          const long long j = off + q;
          if (j < g.R_cap) {
            P.parents[j] = i;
            lab_new[j] = lab_old[i];
          }
        }
      unsigned int pending = __ballot_sync(0xffffffffu, big);
      while (pending) {
        const int src = __ffs(pending) - 1;
        pending &= pending - 1;
        const long long o = __shfl_sync(0xffffffffu, off, src);
        const int cnt = __shfl_sync(0xffffffffu, nb, src);
        const int ii = __shfl_sync(0xffffffffu, i, src);
        const int32_t lab = lab_old[ii];
        for (int q = lane; q < cnt; q += 32) {
          const long long j = o + q;
          if (j < g.R_cap) {
            P.parents[j] = ii;
            lab_new[j] = lab;
          }
        }
      }
      off += nb;
    }
  }
}

__global__ void __launch_bounds__(kCountThreads) k_resample(RunGeom g, PopArgs a, int cur, int t, int32_t* status,
                                                             int spin_limit, int withheld) {
  resample_pop(g, a.p[blockIdx.y], cur, t, status, spin_limit, withheld);
}

// The block's unit: k with off[k] <= blockIdx.x < off[k + 1] (off ascending, n + 1 entries).
__device__ __forceinline__ int group_block_unit(const int32_t* __restrict__ off, int n, int* sh) {
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {  // the last k with off[k] <= b
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    *sh = lo;
  }
  __syncthreads();
  return *sh;
}

// Every unit of a batch: unit k takes blocks off[k] .. off[k+1]-1, one per 1024 slots
// of its capacity; blocks past the old population's tiles take no ticket (the
// tickets stay dense, so every wait is on a block that is running or done).
__global__ void __launch_bounds__(kCountThreads) k_group_resample(const GroupUnit* __restrict__ units,
                                                                   const int32_t* __restrict__ off, int n,
                                                                   const int32_t* __restrict__ round) {
  __shared__ int unit_sh;
  const int k = group_block_unit(off, n, &unit_sh);
  const GroupUnit& u = units[k];
  const int r = *round, t = u.t0 + 1 + r;
  if (t > u.last_t) return;
  const int R_old = u.P.rec[t - 1].R_tilde;
  const int needed = R_old > 0 ? (R_old + kResampleTile - 1) / kResampleTile : 1;
  if ((int)blockIdx.x - off[k] >= needed) return;
  resample_pop(u.g, u.P, u.cur0 ^ (r & 1), t, u.status, kLookbackSpins, -1);
}

// ---------------------------------------------------------------- families (a7)

// Families from the sorted labels: a family is a run of equal labels along the
// slots (labels start as slot numbers and every copy keeps their order), so the
// thread at a run's first slot finds its end (galloping through the labels) and
// knows the family size eta.  Without write_hist: the step's family statistics
// (pa_family.cuh; the last block adds the entropy).  With write_hist: only the
// size histogram m(eta) for the host (lanes of a warp with the same size add with
// one atomic: most families share a few small sizes).
__global__ void __launch_bounds__(256) k_fam_runs(RunGeom g, PopArgs a, int cur, int t, int write_hist) {
  __shared__ long long sh[64];
  const PopDev& P = a.p[blockIdx.y];
  const int R_new = P.rec[t].R_tilde;
  const int32_t* lab = P.labels[cur];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  int eta = 0;
  if (j < R_new) {
    const int32_t l = lab[j];
    if (j == 0 || lab[j - 1] != l) eta = run_end(lab, l, j + 1, R_new) - j;
  }
  if (write_hist) {
    const unsigned peers = __match_any_sync(0xffffffffu, eta);
    if (eta > 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&P.mhist[eta], __popc(peers));
    return;
  }
  FamilyAcc f;
  if (eta > 0) f.add(eta);
  family_size(P, eta, 0xffffffffu);
  family_flush(f, 0xffffffffu, &P.rec[t]);
  family_entropy_last(P, &P.rec[t], R_new, (int)gridDim.x, (int)threadIdx.x, (int)blockDim.x, sh);
}

// Family runs of one rank's slots (sharded runs): the thread at a run's first
// slot finds its end; the first and the last run of the rank's slots may continue
// on the neighbouring ranks, so they go to edge for the host to join; every other
// run is a whole family: eta^2, one family and its size into mhist.
__global__ void __launch_bounds__(256) k_shard_families(RunGeom g, PopDev P, int cur, int t, long long* edge) {
  const int n = P.rec[t].R_tilde;
  const int32_t* lab = P.labels[cur];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  FamilyAcc f;
  if (j < n) {
    const int32_t l = lab[j];
    if (j == 0 || lab[j - 1] != l) {
      const int end = run_end(lab, l, j + 1, n);
      atomicAdd(reinterpret_cast<unsigned long long*>(&edge[5]), 1ull);
      if (j == 0) {
        edge[0] = 1;
        edge[1] = l;
        edge[2] = end;
      }
      if (end == n) {
        edge[3] = l;
        edge[4] = end - j;
      }
      if (j > 0 && end < n) {
        f.add(end - j);
        atomicAdd(&P.mhist[end - j], 1);
      }
    }
  }
  f.s2 = warp_sum(f.s2);
  f.nf = warp_sum(f.nf);
  if ((threadIdx.x & 31) == 0 && f.nf) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&edge[6]), f.s2);
    atomicAdd(reinterpret_cast<unsigned long long*>(&edge[7]), f.nf);
  }
}

// Sum over listed family sizes of m nu ln nu in 128-bit fixed point, one block.
__global__ void __launch_bounds__(1024) k_entropy_of_sizes(const int32_t* eta, const int32_t* m, int K, int R_new,
                                                          long long* out) {
  __shared__ long long sh[64];
  long long hi = 0;
  unsigned long long lo = 0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    long long h;
    unsigned long long l;
    entropy_term(m[k], eta[k], R_new, h, l);
    add128(hi, lo, h, l);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ho = __shfl_xor_sync(0xffffffffu, hi, o);
    const unsigned long long lw = __shfl_xor_sync(0xffffffffu, lo, o);
    add128(hi, lo, ho, lw);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[2 * (threadIdx.x >> 5)] = hi;
    sh[2 * (threadIdx.x >> 5) + 1] = (long long)lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long H = 0;
    unsigned long long Lo = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) add128(H, Lo, sh[2 * w], (unsigned long long)sh[2 * w + 1]);
    out[0] = H;
    out[1] = (long long)Lo;
  }
}

// ---------------------------------------------------------------- overlap (a8)

// q between slot j of population 0 and slot j of population 1, j < min(R~0, R~1):
// Q = N - 2 (sites that differ); bin = ((Q + N)(B - 1) + N) div 2N.
// Block `blk` of the pairs of populations A, B (256 words of four slots each).
__device__ __forceinline__ void overlap_pops(const RunGeom& g, const PopDev& A, const PopDev& B, int cur, int t,
                                             unsigned long long* qhist, unsigned int* qh, int blk) {
  __shared__ unsigned int small_sh;
  const int pairs = min(A.rec[t].R_tilde, B.rec[t].R_tilde);
  for (int i = threadIdx.x; i < g.q_bins; i += blockDim.x) qh[i] = 0u;
  if (threadIdx.x == 0) small_sh = 0u;
  __syncthreads();
  const int wi = blk * blockDim.x + threadIdx.x;
  if (4 * wi < pairs) {
    const uint32_t* SA = reinterpret_cast<const uint32_t*>(A.spins[cur]);
    const uint32_t* SB = reinterpret_cast<const uint32_t*>(B.spins[cur]);
    const int64_t pw = g.pitch / 4;
    int diff[4] = {0, 0, 0, 0};
    uint32_t acc = 0;
    int since = 0;
    for (int n = 0; n < g.N; ++n) {
      acc += ((SA[n * pw + wi] ^ SB[n * pw + wi]) >> 1) & 0x01010101u;
      if (++since == 255) {
#pragma unroll
        for (int b = 0; b < 4; ++b) diff[b] += (acc >> (8 * b)) & 0xFFu;
        acc = 0;
        since = 0;
      }
    }
    unsigned int small = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      diff[b] += (acc >> (8 * b)) & 0xFFu;
      if (4 * wi + b < pairs) {
        const long long Q = (long long)g.N - 2LL * diff[b];
        const long long bin = ((Q + g.N) * (long long)(g.q_bins - 1) + g.N) / (2LL * g.N);
        atomicAdd(&qh[bin], 1u);
        const long long aq = Q < 0 ? -Q : Q;
        small += (5 * aq <= g.N) ? 1u : 0u;
      }
    }
    if (small) atomicAdd(&small_sh, small);
  }
  __syncthreads();
  unsigned long long* row = qhist + (size_t)t * g.q_bins;
  for (int i = threadIdx.x; i < g.q_bins; i += blockDim.x)
    if (qh[i]) atomicAdd(&row[i], (unsigned long long)qh[i]);
  if (threadIdx.x == 0) {
    if (small_sh) atomicAdd(&A.rec[t].q_small, (unsigned long long)small_sh);
    if (blk == 0) A.rec[t].q_pairs = (unsigned long long)pairs;
  }
}

__global__ void k_overlap(RunGeom g, PopArgs a, int cur, int t, unsigned long long* qhist) {
  extern __shared__ unsigned int qh[];
  overlap_pops(g, a.p[0], a.p[1], cur, t, qhist, qh, (int)blockIdx.x);
}

__global__ void k_group_overlap(const GroupUnit* __restrict__ units, const GroupPair* __restrict__ pairs,
                                const int32_t* __restrict__ off, int n, const int32_t* __restrict__ round) {
  extern __shared__ unsigned int qh[];
  __shared__ int pair_sh;
  const int k = group_block_unit(off, n, &pair_sh);
  const GroupPair& pr = pairs[k];
  const GroupUnit& a = units[pr.u0];
  const int r = *round, t = a.t0 + 1 + r;
  if (t > a.last_t) return;
  overlap_pops(a.g, a.P, units[pr.u1].P, a.cur0 ^ ((r + 1) & 1), t, pr.qhist, qh, (int)blockIdx.x - off[k]);
}

__global__ void k_group_advance(int32_t* round) { *round += 1; }

// ---------------------------------------------------------------- launchers

static inline int grid_for(int64_t n, int per) { return (int)((n + per - 1) / per); }

int launch_init_couplings(const RunGeom& g, uint64_t disorder_seed, int8_t* J, uint32_t* jtab, void* stream) {
  const uint32_t k0 = (uint32_t)(disorder_seed & 0xffffffffu);
  const uint32_t k1 = (uint32_t)(disorder_seed >> 32) | (kCouplings << 28);
  k_init_couplings<<<grid_for(g.N, 128), 128, 0, (cudaStream_t)stream>>>(g.N, k0, k1, J, jtab);
  return (int)cudaGetLastError();
}

int launch_init_population(const RunGeom& g, PopDev* pops, int cur, void* stream) {
  const int64_t total = (g.pitch / 4) * g.N;
  dim3 grid(grid_for(total, 256), g.n_pop);
  k_init_population<<<grid, 256, 0, (cudaStream_t)stream>>>(g, pack(pops, g.n_pop), cur);
  return (int)cudaGetLastError();
}

int launch_levels_and_hist(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, int t, void* stream) {
  dim3 grid(grid_for(g.pitch / 4, 128), g.n_pop);
  k_levels_and_hist<<<grid, 128, 0, (cudaStream_t)stream>>>(g, pack(pops, g.n_pop), cur, jtab, t);
  return (int)cudaGetLastError();
}

int launch_reweight(const RunGeom& g, PopDev* pops, const double* w, int t, void* stream) {
  const bool in_smem = g.n_levels <= 3 * kMaxL * kMaxL * kMaxL + 1;  // every lattice of the shared-memory sweep
  const size_t smem = in_smem ? sizeof(int) * (size_t)g.n_levels : 0;
  if (smem > 48 * 1024) {
    static std::atomic<int> done[64];
    const cudaError_t e = smem_limit_once(k_reweight, (int)(sizeof(int) * (3 * kMaxL * kMaxL * kMaxL + 1)), done);
    if (e != cudaSuccess) return (int)e;
  }
  k_reweight<<<g.n_pop, 1024, smem, (cudaStream_t)stream>>>(g, pack(pops, g.n_pop), w, t, in_smem ? 1 : 0);
  return (int)cudaGetLastError();
}

int launch_resample(const RunGeom& g, PopDev* pops, int cur, int t, int32_t* status, const LookbackTest& test,
                    void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  PopArgs a = pack(pops, g.n_pop);
  // the tile ticket was reset by k_reweight, which runs just before on this stream
  const unsigned tiles = (unsigned)((g.R_cap + kResampleTile - 1) / kResampleTile);  // <= n_count_blocks entries
  const int spin_limit = test.spins > 0 ? test.spins : kLookbackSpins;
  k_resample<<<dim3(tiles, g.n_pop), kCountThreads, 0, s>>>(g, a, cur, t, status, spin_limit, test.withheld_tile);
  return (int)cudaGetLastError();
}

int launch_scan_scatter(const RunGeom& g, PopDev* pops, int cur, int t, int32_t* status, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  PopArgs a = pack(pops, g.n_pop);
  k_scan_blocks<<<g.n_pop, 1024, 0, s>>>(g, a, t, status);
  k_scatter<<<dim3(g.n_count_blocks, g.n_pop), kCountThreads, 0, s>>>(g, a, cur, t);
  return (int)cudaGetLastError();
}

int launch_families(const RunGeom& g, PopDev* pops, int cur, int t, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  PopArgs a = pack(pops, g.n_pop);
  k_fam_runs<<<dim3(grid_for(g.R_cap, 256), g.n_pop), 256, 0, s>>>(g, a, cur, t, 0);
  return (int)cudaGetLastError();
}

int launch_shard_families(const RunGeom& g, PopDev* pops, int pop, int cur, int t, long long* edge, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(edge, 0, sizeof(long long) * 8, s);
  cudaMemsetAsync(pops[pop].mhist, 0, sizeof(int32_t) * ((size_t)g.R_cap + 1), s);
  k_shard_families<<<grid_for(g.R_cap, 256), 256, 0, s>>>(g, pops[pop], cur, t, edge);
  return (int)cudaGetLastError();
}

int launch_entropy_of_sizes(const int32_t* eta, const int32_t* m, int K, int R_new, long long* out, void* stream) {
  k_entropy_of_sizes<<<1, 1024, 0, (cudaStream_t)stream>>>(eta, m, K, R_new, out);
  return (int)cudaGetLastError();
}

int launch_family_hist(const RunGeom& g, PopDev* pops, int pop, int cur, int t, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  PopArgs a = pack(pops + pop, 1);
  cudaMemsetAsync(pops[pop].mhist, 0, sizeof(int32_t) * ((size_t)g.R_cap + 1), s);
  k_fam_runs<<<dim3(grid_for(g.R_cap, 256), 1), 256, 0, s>>>(g, a, cur, t, 1);
  return (int)cudaGetLastError();
}

int launch_group_reweight(const GroupUnit* units, int n_units, int max_levels, const int32_t* round, void* stream) {
  const size_t smem = sizeof(int) * (size_t)max_levels;
  if (smem > 48 * 1024) {
    static std::atomic<int> done[64];
    const cudaError_t e =
        smem_limit_once(k_group_reweight, (int)(sizeof(int) * (3 * kMaxL * kMaxL * kMaxL + 1)), done);
    if (e != cudaSuccess) return (int)e;
  }
  k_group_reweight<<<n_units, 1024, smem, (cudaStream_t)stream>>>(units, round);
  return (int)cudaGetLastError();
}

int launch_group_resample(const GroupUnit* units, const int32_t* off, int n_units, int n_blocks, const int32_t* round,
                          void* stream) {
  k_group_resample<<<n_blocks, kCountThreads, 0, (cudaStream_t)stream>>>(units, off, n_units, round);
  return (int)cudaGetLastError();
}

int launch_group_overlap(const GroupUnit* units, const GroupPair* pairs, const int32_t* off, int n_pairs,
                         int n_blocks, int max_bins, const int32_t* round, void* stream) {
  if (n_pairs == 0) return 0;
  k_group_overlap<<<n_blocks, 256, sizeof(unsigned int) * (size_t)max_bins, (cudaStream_t)stream>>>(units, pairs, off,
                                                                                                      n_pairs, round);
  return (int)cudaGetLastError();
}

int launch_group_advance(int32_t* round, void* stream) {
  k_group_advance<<<1, 1, 0, (cudaStream_t)stream>>>(round);
  return (int)cudaGetLastError();
}

int launch_overlap(const RunGeom& g, PopDev* pops, int cur, int t, unsigned long long* qhist, void* stream) {
  if (g.n_pop != 2) return 0;
  const size_t smem = sizeof(unsigned int) * (size_t)g.q_bins;
  k_overlap<<<grid_for(g.pitch / 4, 256), 256, smem, (cudaStream_t)stream>>>(g, pack(pops, 2), cur, t, qhist);
  return (int)cudaGetLastError();
}

}  // namespace pa
