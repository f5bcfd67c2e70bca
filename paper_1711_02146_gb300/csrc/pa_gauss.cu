// pa_gauss.cu — the Gaussian-coupling model (§II.A: J ~ N(0,1)): initial
// energies, resampling from per-replica weights, energy moments and the link
// overlap.  (Its sweep kernel, k_sweep_g, lives with the other sweep kernels.)
//
// Couplings and energies are fixed point (units of 2^-20, couplings clamped to
// [-5, 5]), so energies, their sums and the link overlap are exact integers and
// every floating-point decision has one definition shared with the oracle:
//   - weight of old slot i: w_i = (T2[d >> 24] * T1[(d >> 12) & 4095]) * T0[d & 4095]
//     with d = E_i - E_min and host tables T_k[m] = exp(-dbeta m 2^(12k) 2^-20);
//   - S' = sum_i w_i and the culling sum sum_i (1 - tau_i)_+ in a fixed order:
//     groups of 256 values (zero-padded) each by a binary tree, the group totals
//     again in groups of 256, until one value remains;
//   - tau_i = R w_i / S', n_i = floor(tau_i) + [r_i < 2^32 frac(tau_i)] (§II).
#include <cuda_runtime.h>

#include <algorithm>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

struct GArgs {
  PopDev p[2];
};

GArgs gpack(const PopDev* pops, int n_pop) {
  GArgs a;
  for (int i = 0; i < n_pop && i < 2; ++i) a.p[i] = pops[i];
  return a;
}

__host__ __device__ inline int blocks_for(long long n, int per) { return (int)((n + per - 1) / per); }

constexpr uint32_t kBit1 = 0x02020202u;  // bit 1 of each byte: the two int8 spins differ

// ---------------------------------------------------------------- initial energies

// E_j = -sum_bonds J s s = -Jtot + 2 sum over antiparallel bonds of J, for the
// four slots of one 32-bit word of every site row (int8 spins, site-major).
__global__ void k_g_energy_init(RunGeom g, GArgs a, int cur, const int32_t* __restrict__ Jq) {
  const PopDev& P = a.p[blockIdx.y];
  const int R = P.rec[0].R_tilde;
  const int wi = blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * wi >= R) return;
  const int L = g.L;
  const uint32_t* S = reinterpret_cast<const uint32_t*>(P.spins[cur]);
  const int64_t pw = g.pitch / 4;
  long long anti[4] = {0, 0, 0, 0}, jtot = 0;
  for (int n = 0; n < g.N; ++n) {
    const int x = n % L, y = (n / L) % L, z = n / (L * L);
    const int nb[3] = {(x + 1 == L ? 0 : x + 1) + L * (y + L * z), x + L * ((y + 1 == L ? 0 : y + 1) + L * z),
                       x + L * (y + L * (z + 1 == L ? 0 : z + 1))};
    const uint32_t s = S[n * pw + wi];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long J = Jq[3 * n + d];
      jtot += J;
      const uint32_t x4 = (s ^ S[nb[d] * pw + wi]) & kBit1;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if ((x4 >> (8 * b + 1)) & 1u) anti[b] += J;
    }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = 4 * wi + b;
    if (j < R) P.E64[j] = -jtot + 2 * anti[b];
  }
}

// Opens the records of step t (what k_g_weights does for t >= 1).
__global__ void k_g_open(GArgs a, int t) {
  GRec& r = a.p[threadIdx.x].grec[t];
  r.E_min = 0x7fffffffffffffffLL;
  r.E0 = 0;
  r.sum_E = 0;
  r.sum_E2_lo = r.sum_E2_hi = 0;
  r.n_at_E0 = 0;
  r.ql_sum = 0;
}

// ---------------------------------------------------------------- resampling

// Sum of a[0..256) of shared memory by the fixed binary tree; result in a[0].
__device__ __forceinline__ void chunk_tree(double* a) {
  for (int h = kChunk / 2; h >= 1; h >>= 1) {
    if ((int)threadIdx.x < h) a[threadIdx.x] = __dadd_rn(a[threadIdx.x], a[threadIdx.x + h]);
    __syncthreads();
  }
}

// Whether this block is the last of the launch's n_blocks blocks (of its
// population) to finish: each block, once its chunk total is written, counts
// itself on the ticket; the last one sums every total (tree_total) and resets it.
__device__ __forceinline__ bool last_block_done(int32_t* ticket, int n_blocks) {
  __shared__ int last;
  __syncthreads();  // the block's chunk total is written
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1) == n_blocks - 1;
    if (last) *ticket = 0;
  }
  __syncthreads();
  return last;
}

// The chunk_tree sum of 256 values held by one warp, lane l holding entries l + 32 k
// in v[k]: the tree's steps 128, 64 and 32 are additions within a lane and 16 .. 1
// additions across lanes, each pair added in the tree's order.  The sum in lane 0.
// warp_group_sum: the same for the entries src[base, base + 256) (zeros from n on).
__device__ __forceinline__ double group8(double* v) {
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = __dadd_rn(v[k], v[k + 4]);
  v[0] = __dadd_rn(v[0], v[2]);
  v[1] = __dadd_rn(v[1], v[3]);
  v[0] = __dadd_rn(v[0], v[1]);
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) v[0] = __dadd_rn(v[0], __shfl_down_sync(0xffffffffu, v[0], h));
  return v[0];
}

__device__ __forceinline__ double warp_group_sum(const double* src, long long base, int n) {
  const int lane = threadIdx.x & 31;
  double v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const long long i = base + lane + 32 * k;
    v[k] = i < n ? __ldcg(src + i) : 0.0;
  }
  return group8(v);
}

// The sum of the n_chunks chunk totals at the start of part by a fixed tree, in
// this one block: each level's entries in groups of 256 (zeros past its last
// entry) added by the chunk_tree order (warp_group_sum, one warp per group), the
// group sums stored after the level's entries in part as the next level, until one
// group is left.  The order depends only on n_chunks, so every launch adds in the
// same order.  The total in thread 0.
__device__ double tree_total(double* part, int n_chunks) {
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, n_warps = blockDim.x >> 5;
  long long off = 0;
  int n = n_chunks;
  double total = 0.0;
  for (;;) {
    const int nb = (n + kChunk - 1) / kChunk;
    for (int b = warp; b < nb; b += n_warps) {
      const double v = warp_group_sum(part + off, (long long)b * kChunk, n);
      if (lane == 0) {
        if (nb == 1)
          total = v;
        else
          part[off + n + b] = v;
      }
    }
    __syncthreads();
    if (nb == 1) break;
    off += n;
    n = nb;
  }
  return total;
}

// Weights of the old slots of step t-1 and their chunk partial sums; the last
// block to finish adds the partial sums into S'.  Block 0 also opens the records
// of step t.  A trial of the bisection whose halvings have reached their fixed
// point (*skip != 0, see k_g_tau) does nothing.
__global__ void __launch_bounds__(kChunk) k_g_weights(RunGeom g, GArgs a, int t, const double* __restrict__ T,
                                                     const double* skip) {
  __shared__ double sh[kChunk];
  if (skip && *skip != 0.0) return;
  PopDev& P = a.p[blockIdx.y];
  const int R_old = P.rec[t - 1].R_tilde;
  const long long Emin = P.grec[t - 1].E_min;
  const int i = blockIdx.x * kChunk + threadIdx.x;
  double w = 0.0;
  if (i < R_old) {
    const long long d = P.E64[i] - Emin;
    w = __dmul_rn(__dmul_rn(T[8192 + (d >> 24)], T[4096 + ((d >> 12) & 4095)]), T[d & 4095]);
    P.w[i] = w;
  }
  sh[threadIdx.x] = w;
  __syncthreads();
  chunk_tree(sh);
  if (threadIdx.x == 0) P.part[blockIdx.x] = sh[0];
  if (last_block_done(P.ticket, (int)gridDim.x)) {
    const double S = tree_total(P.part, (int)gridDim.x);
    if (threadIdx.x == 0) P.rec[t].S_prime = S;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.rec[t].R_prev = R_old;
    GRec& r = P.grec[t];
    r.E_min = 0x7fffffffffffffffLL;
    r.E0 = 0;
    r.sum_E = 0;
    r.sum_E2_lo = r.sum_E2_hi = 0;
    r.n_at_E0 = 0;
    r.ql_sum = 0;
  }
}

// tau_i = R w_i / S', its floor and 2^32-scaled fraction (not in a trial of the
// adaptive schedule, which needs only the culling fraction), and the chunk partial
// sums of S' (1 - tau_i)_+ = (S' - R w_i)_+; the last block to finish adds them and
// divides by S' R into the expected culling fraction (Eq. eq_num_elim: the same sum
// with one division instead of one per replica).  In the adaptive bisection
// (b = {lo, hi, mid}, population 0 only) that block also takes the halving's
// decision: mid becomes lo when the fraction does not exceed the target, else hi,
// and the next midpoint is 0.5 (lo + hi) (the host's arithmetic, rounded the same
// way).  b[3] becomes 1 once that midpoint equals hi, a point already rejected, or
// lo > 0, a point already accepted: every later halving then evaluates the same
// point again, takes the same decision and leaves {lo, hi, mid} as they are, so the
// remaining trials are skipped (identical results, fewer launches doing work).
__global__ void __launch_bounds__(kChunk) k_g_tau(RunGeom g, GArgs a, int t, double* b, double target,
                                                 int trial) {
  __shared__ double sh[kChunk];
  if (b && b[3] != 0.0) return;
  PopDev& P = a.p[blockIdx.y];
  const int R_old = P.rec[t - 1].R_tilde;
  const double S = P.rec[t].S_prime;
  const int i = blockIdx.x * kChunk + threadIdx.x;
  double c = 0.0;
  if (i < R_old) {
    const double rw = __dmul_rn((double)g.R, P.w[i]);
    if (!trial) {
      const double tau = __ddiv_rn(rw, S);
      const double f = floor(tau);
      P.gfl[i] = (int32_t)f;
      P.gthr[i] = __double2uint_rz(__dmul_rn(__dsub_rn(tau, f), 4294967296.0));
    }
    c = rw < S ? __dsub_rn(S, rw) : 0.0;
  }
  sh[threadIdx.x] = c;
  __syncthreads();
  chunk_tree(sh);
  if (threadIdx.x == 0) P.part[blockIdx.x] = sh[0];
  if (last_block_done(P.ticket, (int)gridDim.x)) {
    const double total = tree_total(P.part, (int)gridDim.x);
    if (threadIdx.x == 0) {
      const double e = __ddiv_rn(__ddiv_rn(total, S), (double)g.R);
      P.rec[t].eps_expected = e;
      if (b) {
        if (e <= target)
          b[0] = b[2];
        else
          b[1] = b[2];
        b[2] = __dmul_rn(0.5, __dadd_rn(b[0], b[1]));
        b[3] = (b[2] == b[1] || (b[2] == b[0] && b[0] > 0.0)) ? 1.0 : 0.0;
      }
    }
  }
}

// Copy numbers n_i = fl_i + [r_i < thr_i], r_i = word (i & 3) of Philox at counter
// (i >> 2, 0, 0, t) keyed by (run seed, resampling, population); block totals
// feed the scan of the ±1 path.
__global__ void __launch_bounds__(kCountThreads) k_g_counts(RunGeom g, GArgs a, int t) {
  __shared__ int red[kCountThreads / 32];
  PopDev& P = a.p[blockIdx.y];
  const int R_old = P.rec[t - 1].R_tilde;
  const int i0 = blockIdx.x * kSlotsPerCountBlock + 4 * threadIdx.x;
  int sum = 0, cul = 0;
  if (i0 < R_old) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)(i0 >> 2), 0u, 0u, (uint32_t)t), P.key_res[0], P.key_res[1]);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + b;
      if (i < R_old) {
        const int n = P.gfl[i] + (word_of(r, b) < P.gthr[i] ? 1 : 0);
        P.counts[i] = n;
        sum += n;
        cul += (n == 0);
      }
    }
  }
  sum = warp_sum(sum);
  cul = warp_sum(cul);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = sum;
    if (cul) atomicAdd(&P.rec[t].culled, cul);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int k = 0; k < kCountThreads / 32; ++k) s += red[k];
    P.blocksums[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------- adaptive schedule

// Weight tables T_k[m] = exp(-dbeta m 2^(12k) 2^-20) (T0 | T1 | T2, kGTableWeights
// entries) for dbeta = *dbeta_dev, or dbeta_val when dbeta_dev is null: the
// adaptive schedule's trials and its chosen step build their tables here, so a
// trial and the resampling that follows it use the same weights.  Nothing is
// written when *skip != 0 (a bisection at its fixed point, see k_g_tau).
__device__ __forceinline__ double g_table_entry(double db, int m) {
  const long long q = m < 4096 ? (long long)m : m < 8192 ? (long long)(m - 4096) << 12 : (long long)(m - 8192) << 24;
  return exp(-__dmul_rn(db, __dmul_rn((double)q, 0x1p-20)));
}

__global__ void k_g_tables(const double* __restrict__ dbeta_dev, double dbeta_val, double* T, const double* skip) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= kGTableWeights || (skip && *skip != 0.0)) return;
  T[m] = g_table_entry(dbeta_dev ? *dbeta_dev : dbeta_val, m);
}

// The whole bisection in one cooperative launch (every block resident, blocks of
// kBisectThreads): each halving is one pass over the old population for the
// weights of mid and their chunk partial sums, a grid barrier whose last block to
// arrive adds the partial sums (block_total, the order of tree_total) into S', a
// pass for the culling terms (S' - R w_i)_+ and their chunk partial sums, and a
// second such barrier for their total; every block then takes the same decision.
// The weight tables of the two possible next midpoints are built during the second
// pass, into the two table sets not in use, T2 only up to the entry of the largest
// d = E_i - E_min (found once, before the first halving).  The values, sums and
// decisions are those of the launch-per-trial path (k_g_tables, k_g_weights,
// k_g_tau), so both give the same lo, hi and mid.
constexpr int kBisectThreads = 256;
constexpr int kBisectWarps = kBisectThreads / 32;
constexpr int kBisectMaxChunks = kChunk * kChunk;  // block_total keeps two tree levels
constexpr unsigned kBarrierSpins = 1u << 22;       // polls of one barrier wait (about 0.5 s at most)
// words of the barrier block: arrivals, generation, error, largest d, S', culling sum
enum { kBarArrive, kBarGen, kBarError, kBarDmax, kBarS, kBarCull, kBarWords = 8 };

// tree_total of the n partial sums part[0, n) (n <= kBisectMaxChunks), computed by
// this block alone: the first level's groups by its warps, the second level (at
// most 256 group sums) from shared memory by warp 0.  The total in thread 0.
__device__ double block_total(const double* part, int n, double* lvl) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = (n + kChunk - 1) / kChunk;
  for (int b = warp; b < nb; b += kBisectWarps) {
    const double v = warp_group_sum(part, (long long)b * kChunk, n);
    if (lane == 0) lvl[b] = v;
  }
  __syncthreads();
  double x = 0.0;
  if (warp == 0) {
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = lane + 32 * k;
      v[k] = i < nb ? lvl[i] : 0.0;
    }
    x = nb == 1 ? lvl[0] : group8(v);
  }
  __syncthreads();
  return x;
}

// Grid barrier of a cooperative launch: the last block to arrive resets the count
// and advances the generation, the others poll it at most `spins` times.  With
// part, that last block first stores block_total(part, n) in bar[slot].  A wait that
// runs out records the error, after which every barrier returns at once (false) and
// the launch ends with the error set.  A block with withhold set waits without
// arriving (a test of that path: the waits then run out).
__device__ bool grid_barrier(unsigned long long* bar, unsigned spins_max, bool withhold = false,
                             const double* part = nullptr, int n = 0, int slot = 0, double* lvl = nullptr) {
  __shared__ int state;  // 0: wait, 1: last to arrive, -1: error
  volatile unsigned long long* vb = bar;
  unsigned long long gen = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int st = vb[kBarError] == 0ull ? 0 : -1;
    if (st == 0) {
      gen = vb[kBarGen];
      __threadfence();
      if (!withhold && atomicAdd(&bar[kBarArrive], 1ull) == (unsigned long long)gridDim.x - 1ull) st = 1;
    }
    state = st;
  }
  __syncthreads();
  if (state == 1 && part) {
    const double x = block_total(part, n, lvl);
    if (threadIdx.x == 0) vb[slot] = (unsigned long long)__double_as_longlong(x);
  }
  if (threadIdx.x == 0) {
    if (state == 1) {
      __threadfence();
      atomicExch(&bar[kBarArrive], 0ull);
      __threadfence();
      atomicAdd(&bar[kBarGen], 1ull);
    } else if (state == 0) {
      unsigned spins = 0;
      while (vb[kBarGen] == gen && vb[kBarError] == 0ull && ++spins < spins_max) __nanosleep(64);
      if (vb[kBarGen] == gen) {
        atomicExch(&bar[kBarError], 1ull);
        state = -1;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return state >= 0;
}

__device__ __forceinline__ double bar_double(const unsigned long long* bar, int slot) {
  return __longlong_as_double((long long)((volatile const unsigned long long*)bar)[slot]);
}

struct BisectArgs {
  PopDev P;                 // population 0 decides the step
  double* b;                // {lo, hi, mid, state}: in, and out (state 1 done, -1 a barrier wait ran out)
  double* T;                // three sets of kGTableWeights table entries
  double* part1;            // [n_chunks] chunk partial sums of the culling terms (those of the weights in P.part)
  unsigned long long* bar;  // kBarWords words, zero at launch
  unsigned spins;           // polls of a barrier wait
  int withheld;             // block that does not arrive at the first barrier (-1: none; tests)
  int t, R, halvings;
  double target;
};

__global__ void __launch_bounds__(kBisectThreads, 4) k_g_bisect(BisectArgs a) {
  __shared__ double lvl[kChunk];
  const PopDev& P = a.P;
  const int R_old = P.rec[a.t - 1].R_tilde;
  const long long Emin = P.grec[a.t - 1].E_min;
  const int nch = (R_old + kChunk - 1) / kChunk;
  const int lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * kBisectWarps + (threadIdx.x >> 5);
  const int n_warps = gridDim.x * kBisectWarps;
  const int gtid = blockIdx.x * kBisectThreads + threadIdx.x;
  const int n_threads = gridDim.x * kBisectThreads;
  const double R = (double)a.R;
  double lo = a.b[0], hi = a.b[1], mid = a.b[2];
  unsigned long long dmax = 0;  // the largest d: T2 beyond its entry is never read
  for (int i = gtid; i < R_old; i += n_threads) {
    const unsigned long long d = (unsigned long long)(P.E64[i] - Emin);
    dmax = d > dmax ? d : dmax;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_down_sync(0xffffffffu, dmax, o);
    dmax = x > dmax ? x : dmax;
  }
  if (lane == 0 && dmax) atomicMax(&a.bar[kBarDmax], dmax);
  bool ok = grid_barrier(a.bar, a.spins, (int)blockIdx.x == a.withheld);
  const int n_tab = 8192 + (int)min(8191ull, ((volatile unsigned long long*)a.bar)[kBarDmax] >> 24) + 1;
  for (int m = gtid; m < n_tab; m += n_threads) a.T[m] = g_table_entry(mid, m);
  int cur = 0;
  ok = ok && grid_barrier(a.bar, a.spins);
  for (int h = 0; h < a.halvings && ok; ++h) {
    const double* Tc = a.T + (size_t)cur * kGTableWeights;
    for (int c = gwarp; c < nch; c += n_warps) {  // weights of mid and their chunk sums
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = c * kChunk + lane + 32 * k;
        v[k] = 0.0;
        if (i < R_old) {
          const long long d = P.E64[i] - Emin;
          v[k] = __dmul_rn(__dmul_rn(__ldcg(Tc + 8192 + (d >> 24)), __ldcg(Tc + 4096 + ((d >> 12) & 4095))),
                           __ldcg(Tc + (d & 4095)));
          __stcg(P.w + i, v[k]);
        }
      }
      const double sum = group8(v);
      if (lane == 0) __stcg(P.part + c, sum);
    }
    if (!grid_barrier(a.bar, a.spins, false, P.part, nch, kBarS, lvl)) break;
    const double S = bar_double(a.bar, kBarS);
    const long long S_bits = __double_as_longlong(S);
    const int s_acc = cur == 2 ? 0 : cur + 1, s_rej = cur == 0 ? 2 : cur - 1;
    const double m_acc = __dmul_rn(0.5, __dadd_rn(mid, hi)), m_rej = __dmul_rn(0.5, __dadd_rn(lo, mid));
    for (int m = gtid; m < 2 * n_tab; m += n_threads) {  // both possible next tables
      const bool acc = m < n_tab;
      const int e = acc ? m : m - n_tab;
      a.T[(size_t)(acc ? s_acc : s_rej) * kGTableWeights + e] = g_table_entry(acc ? m_acc : m_rej, e);
    }
    for (int c = gwarp; c < nch; c += n_warps) {  // culling terms and their chunk sums
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = c * kChunk + lane + 32 * k;
        v[k] = 0.0;
        if (i < R_old) {
          // rw < S' compared as the bit patterns of two non-negative doubles (an
          // integer comparison, the same order)
          const double rw = __dmul_rn(R, __ldcg(P.w + i));
          if (__double_as_longlong(rw) < S_bits) v[k] = __dsub_rn(S, rw);
        }
      }
      const double sum = group8(v);
      if (lane == 0) __stcg(a.part1 + c, sum);
    }
    if (!grid_barrier(a.bar, a.spins, false, a.part1, nch, kBarCull, lvl)) break;
    const double e = __ddiv_rn(__ddiv_rn(bar_double(a.bar, kBarCull), S), R);
    if (e <= a.target) {
      lo = mid;
      cur = s_acc;
    } else {
      hi = mid;
      cur = s_rej;
    }
    mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
    // the fixed point of k_g_tau: every later halving evaluates a point already decided
    if (mid == hi || (mid == lo && lo > 0.0)) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.b[0] = lo;
    a.b[1] = hi;
    a.b[2] = mid;
    a.b[3] = ((volatile unsigned long long*)a.bar)[kBarError] != 0ull ? -1.0 : 1.0;
  }
}

// ---------------------------------------------------------------- measurement

constexpr int kMeasureThreads = 256;
constexpr int kMeasurePerBlock = 4096;

// Lowest energy, exact sum, and 128-bit partial sums of E^2 of the step-t population.
__global__ void __launch_bounds__(kMeasureThreads) k_g_moments(RunGeom g, GArgs a, int t) {
  __shared__ long long smin[kMeasureThreads / 32], ssum[kMeasureThreads / 32];
  __shared__ unsigned long long s2lo[kMeasureThreads / 32], s2hi[kMeasureThreads / 32];
  PopDev& P = a.p[blockIdx.y];
  const int R = P.rec[t].R_tilde;
  long long mn = 0x7fffffffffffffffLL, sm = 0;
  unsigned __int128 s2 = 0;
  const int base = blockIdx.x * kMeasurePerBlock;
  for (int k = threadIdx.x; k < kMeasurePerBlock; k += kMeasureThreads) {
    const int j = base + k;
    if (j < R) {
      const long long E = P.E64[j];
      mn = E < mn ? E : mn;
      sm += E;
      s2 += (unsigned __int128)(E < 0 ? -E : E) * (unsigned __int128)(E < 0 ? -E : E);
    }
  }
  unsigned long long lo = (unsigned long long)s2, hi = (unsigned long long)(s2 >> 64);
  for (int o = 16; o > 0; o >>= 1) {
    const long long m2 = __shfl_down_sync(0xffffffffu, mn, o);
    mn = m2 < mn ? m2 : mn;
    sm += __shfl_down_sync(0xffffffffu, sm, o);
    const unsigned long long lo2 = __shfl_down_sync(0xffffffffu, lo, o);
    const unsigned long long hi2 = __shfl_down_sync(0xffffffffu, hi, o);
    const unsigned long long nl = lo + lo2;
    hi = hi + hi2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  const int wv = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    smin[wv] = mn;
    ssum[wv] = sm;
    s2lo[wv] = lo;
    s2hi[wv] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned __int128 tot = 0;
    for (int k = 0; k < kMeasureThreads / 32; ++k) {
      mn = smin[k] < mn ? smin[k] : mn;
      tot += ((unsigned __int128)s2hi[k] << 64) | s2lo[k];
    }
    long long st = 0;
    for (int k = 0; k < kMeasureThreads / 32; ++k) st += ssum[k];
    atomicMin(&P.grec[t].E_min, mn);
    atomicAdd(reinterpret_cast<unsigned long long*>(&P.grec[t].sum_E), (unsigned long long)st);
    P.e2part[2 * blockIdx.x] = (unsigned long long)tot;
    P.e2part[2 * blockIdx.x + 1] = (unsigned long long)(tot >> 64);
  }
}

// One thread per population: the exact sum of E^2 and E0 = min(E0 of t-1, E_min of t).
__global__ void k_g_finish(RunGeom g, GArgs a, int t) {
  PopDev& P = a.p[threadIdx.x];
  const int R = P.rec[t].R_tilde;
  GRec& r = P.grec[t];
  unsigned __int128 s2 = 0;
  for (int b = 0; b < blocks_for(R, kMeasurePerBlock); ++b)
    s2 += ((unsigned __int128)P.e2part[2 * b + 1] << 64) | P.e2part[2 * b];
  r.sum_E2_lo = (unsigned long long)s2;
  r.sum_E2_hi = (unsigned long long)(s2 >> 64);
  r.E0 = (t == 0 || r.E_min < P.grec[t - 1].E0) ? r.E_min : P.grec[t - 1].E0;
  r.n_at_E0 = 0;
}

// Replicas at E0.
__global__ void __launch_bounds__(kMeasureThreads) k_g_count_E0(RunGeom g, GArgs a, int t) {
  PopDev& P = a.p[blockIdx.y];
  const int R = P.rec[t].R_tilde;
  const long long E0 = P.grec[t].E0;
  const int base = blockIdx.x * kMeasurePerBlock;
  long long c = 0;
  for (int k = threadIdx.x; k < kMeasurePerBlock; k += kMeasureThreads) {
    const int j = base + k;
    if (j < R) c += P.E64[j] == E0;
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c)
    atomicAdd(reinterpret_cast<unsigned long long*>(&P.grec[t].n_at_E0), (unsigned long long)c);
}

// Link overlap (Eq. ql) between slot j of the two populations, four pairs per
// thread: with c = s1 s2 per site, QL = sum over bonds of c_n c_m = N_b - 2
// (bonds whose c differ); histogram bin ((QL + N_b)(B - 1) + N_b) div 2N_b.
__global__ void k_g_link(RunGeom g, GArgs a, int cur, int t, unsigned long long* qlhist) {
  extern __shared__ unsigned int qh[];
  __shared__ long long ssum;
  const PopDev& A = a.p[0];
  const PopDev& B = a.p[1];
  const int pairs = min(A.rec[t].R_tilde, B.rec[t].R_tilde);
  for (int i = threadIdx.x; i < g.q_bins; i += blockDim.x) qh[i] = 0u;
  if (threadIdx.x == 0) ssum = 0;
  __syncthreads();
  const int wi = blockIdx.x * blockDim.x + threadIdx.x;
  const long long Nb = 3LL * g.N;
  if (4 * wi < pairs) {
    const int L = g.L;
    const uint32_t* SA = reinterpret_cast<const uint32_t*>(A.spins[cur]);
    const uint32_t* SB = reinterpret_cast<const uint32_t*>(B.spins[cur]);
    const int64_t pw = g.pitch / 4;
    int diff[4] = {0, 0, 0, 0};
    uint32_t acc = 0;
    int since = 0;
    for (int n = 0; n < g.N; ++n) {
      const int x = n % L, y = (n / L) % L, z = n / (L * L);
      const int nx = (x + 1 == L ? 0 : x + 1) + L * (y + L * z);
      const int ny = x + L * ((y + 1 == L ? 0 : y + 1) + L * z);
      const int nz = x + L * (y + L * (z + 1 == L ? 0 : z + 1));
      const uint32_t c = SA[n * pw + wi] ^ SB[n * pw + wi];
      acc += ((c ^ SA[nx * pw + wi] ^ SB[nx * pw + wi]) & kBit1) + ((c ^ SA[ny * pw + wi] ^ SB[ny * pw + wi]) & kBit1) +
             ((c ^ SA[nz * pw + wi] ^ SB[nz * pw + wi]) & kBit1);
      if (++since == 40) {
#pragma unroll
        for (int b = 0; b < 4; ++b) diff[b] += (acc >> (8 * b + 1)) & 0x7Fu;
        acc = 0;
        since = 0;
      }
    }
    long long local = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      diff[b] += (acc >> (8 * b + 1)) & 0x7Fu;
      if (4 * wi + b < pairs) {
        const long long QL = Nb - 2LL * diff[b];
        atomicAdd(&qh[((QL + Nb) * (long long)(g.q_bins - 1) + Nb) / (2 * Nb)], 1u);
        local += QL;
      }
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&ssum), (unsigned long long)local);
  }
  __syncthreads();
  unsigned long long* row = qlhist + (size_t)t * g.q_bins;
  for (int i = threadIdx.x; i < g.q_bins; i += blockDim.x)
    if (qh[i]) atomicAdd(&row[i], (unsigned long long)qh[i]);
  if (threadIdx.x == 0 && ssum)
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.p[0].grec[t].ql_sum), (unsigned long long)ssum);
}

}  // namespace

// ---------------------------------------------------------------- launchers

int launch_g_energy_init(const RunGeom& g, PopDev* pops, int cur, const int32_t* Jq, void* stream) {
  dim3 grid(blocks_for(g.pitch / 4, 128), g.n_pop);
  k_g_energy_init<<<grid, 128, 0, (cudaStream_t)stream>>>(g, gpack(pops, g.n_pop), cur, Jq);
  return (int)cudaGetLastError();
}

int launch_g_resample(const RunGeom& g, PopDev* pops, int cur, int t, const double* wtab, int32_t* status,
                      void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  GArgs a = gpack(pops, g.n_pop);
  const dim3 chunks(g.n_chunks, g.n_pop);
  k_g_weights<<<chunks, kChunk, 0, s>>>(g, a, t, wtab, nullptr);
  k_g_tau<<<chunks, kChunk, 0, s>>>(g, a, t, nullptr, 0.0, 0);
  k_g_counts<<<dim3(g.n_count_blocks, g.n_pop), kCountThreads, 0, s>>>(g, a, t);
  const int e = (int)cudaGetLastError();
  return e ? e : launch_scan_scatter(g, pops, cur, t, status, stream);
}

// One trial of the adaptive schedule on population 0; with b, also the bisection's
// halving that follows from it.
static int eps_trial(const RunGeom& g, PopDev* pops, int t, const double* wtab, double* b, double target,
                     cudaStream_t s) {
  RunGeom g1 = g;  // population 0 decides the step
  g1.n_pop = 1;
  GArgs a = gpack(pops, 1);
  const dim3 chunks(g1.n_chunks, 1);
  k_g_weights<<<chunks, kChunk, 0, s>>>(g1, a, t, wtab, b ? b + 3 : nullptr);
  k_g_tau<<<chunks, kChunk, 0, s>>>(g1, a, t, b, target, 1);
  return (int)cudaGetLastError();
}

int launch_g_eps_trial(const RunGeom& g, PopDev* pops, int t, const double* wtab, void* stream) {
  return eps_trial(g, pops, t, wtab, nullptr, 0.0, (cudaStream_t)stream);
}

int launch_g_tables(const double* dbeta_dev, double dbeta_val, double* T, void* stream) {
  k_g_tables<<<blocks_for(kGTableWeights, 256), 256, 0, (cudaStream_t)stream>>>(dbeta_dev, dbeta_val, T, nullptr);
  return (int)cudaGetLastError();
}

int launch_g_bisect(const RunGeom& g, PopDev* pops, int t, double* T, double* b, double target, int halvings,
                    void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  for (int it = 0; it < halvings; ++it) {
    k_g_tables<<<blocks_for(kGTableWeights, 256), 256, 0, s>>>(b + 2, 0.0, T, b + 3);
    const int e = eps_trial(g, pops, t, T, b, target, s);
    if (e) return e;
  }
  return (int)cudaGetLastError();
}

int g_bisect_blocks(const RunGeom& g) {
  if (g.n_chunks > kBisectMaxChunks) return 0;
  int dev = 0, n_sm = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_g_bisect, kBisectThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int want = blocks_for(g.n_chunks, kBisectWarps);  // one chunk per warp when the device holds them
  return std::max(1, std::min(want, per_sm * n_sm));
}

int launch_g_bisect_fused(const RunGeom& g, PopDev* pops, int t, double* tables, double* part1,
                          unsigned long long* bar, double* b, double target, int halvings, int n_blocks,
                          int withheld, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  BisectArgs a;
  a.P = pops[0];
  a.b = b;
  a.T = tables;
  a.part1 = part1;
  a.bar = bar;
  a.t = t;
  a.R = g.R;
  a.halvings = halvings;
  a.target = target;
  a.withheld = withheld;
  a.spins = withheld >= 0 ? 4096u : kBarrierSpins;
  cudaError_t e = cudaMemsetAsync(bar, 0, kBarWords * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return (int)e;
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)k_g_bisect, dim3((unsigned)n_blocks), dim3(kBisectThreads), args, 0, s);
  return (int)e;
}

int launch_g_measure(const RunGeom& g, PopDev* pops, int cur, int t, unsigned long long* qlhist, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  GArgs a = gpack(pops, g.n_pop);
  if (t == 0) k_g_open<<<1, g.n_pop, 0, s>>>(a, 0);  // step 0 has no resampling to open its records
  k_g_moments<<<dim3(g.n_measure_blocks, g.n_pop), kMeasureThreads, 0, s>>>(g, a, t);
  k_g_finish<<<1, g.n_pop, 0, s>>>(g, a, t);
  k_g_count_E0<<<dim3(g.n_measure_blocks, g.n_pop), kMeasureThreads, 0, s>>>(g, a, t);
  if (g.n_pop == 2) {
    const size_t smem = sizeof(unsigned int) * (size_t)g.q_bins;
    k_g_link<<<blocks_for(g.pitch / 4, 256), 256, smem, s>>>(g, a, cur, t, qlhist);
  }
  return (int)cudaGetLastError();
}

}  // namespace pa
