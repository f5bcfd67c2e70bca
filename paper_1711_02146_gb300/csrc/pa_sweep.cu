// pa_sweep.cu — the Metropolis sweep kernel (the dominant cost of a PA step).
//
// One CTA owns a tile of TJ = 4W consecutive slots of the NEW population and
// all N sites of those replicas in shared memory (W 32-bit words per site row,
// four replicas per word).  It
//   1. gathers each slot's spins from its parent in the old population (the
//      replica copy of the resampling, §II, fused into the load),
//   2. runs S checkerboard Metropolis sweeps at beta_t in shared memory (colour
//      c = (x + y + z) & 1, colour 0 then colour 1; the neighbours of a site all
//      have the other colour, so all sites of one colour update independently),
//   3. counts each replica's unsatisfied bonds (its energy level k) and adds
//      the tile to the level histogram of step t, and
//   4. writes the tile to the new population buffer.
// HBM traffic is one read and one write of the tile per step, whatever S is.
//
// Metropolis rule: flipping s_n costs dE = 2 s_n h_n = 12 - 4u, u = unsatisfied
// bonds at n.  It is taken when u >= 3 (dE <= 0) or when the Philox word r is
// below thr[dE/4 - 1] = floor(2^32 exp(-beta dE)).  r is word (j & 3) of
// Philox4x32-10 at counter (n >> 1, 2s + c, j >> 2, t) keyed by (run_seed,
// Metropolis, population): one call serves the four replicas of a word.
//
// Shared-memory encoding: a spin is one byte, 0x00 for +1 and 0x04 for -1 (HBM
// holds int8 +1 = 0x01 / -1 = 0xFF).  For a bond, s_a ^ s_b ^ Jmask (Jmask =
// 0x04 per byte for J = -1) is 0x04 exactly when the bond is unsatisfied, so the
// byte-wise sum of the six bond terms is 4u, which is also the byte offset of
// u's entry in a 7-word threshold table.
//
// Philox hoisting (same function, fewer multiplies): with counter words
// (h, q, g, t) = (site, half-sweep, word, step), the round-1 and round-2
// products depend either on the site and step only (tabulated once per launch
// in shared memory) or on the thread and half-sweep only (registers), so each
// block costs the 16 wide multiplies of rounds 3..10.
#include <cuda_runtime.h>

#include "pa_device.cuh"
#include "pa_internal.h"

// Threads per CTA of the L = 10 sweep (a multiple of 32 whose row partitions
// divide the 100 rows evenly: 640 = 20 partitions of 5 rows, 800 = 25 of 4).
#ifndef PA_SWEEP_NT_L10
#define PA_SWEEP_NT_L10 640
#endif
// Words per site row of the L = 10 tile (32: 128 replicas, one warp per row;
// 16: 64 replicas, two rows per warp and two CTAs per SM).
#ifndef PA_SWEEP_W_L10
#define PA_SWEEP_W_L10 32
#endif

namespace pa {

constexpr uint32_t kM0 = 0xD2511F53u;
constexpr uint32_t kM1 = 0xCD9E8D57u;
constexpr uint32_t kSpinBit = 0x04040404u;

struct SweepArgs {
  PopDev pop;
  const uint32_t* jtab;  // [N][4] forward-bond masks (0xFEFEFEFE for J = -1)
  int64_t pitch;
  int32_t n_levels;
  int32_t t;
  int32_t cur;
  int32_t n_sweeps;
  uint32_t thr4, thr8, thr12;
  uint32_t k0[10];       // Metropolis round keys of this population
  uint32_t k1[10];
};

// Per-site shared-memory record: the six bond masks of the site, and the
// site/step-dependent parts of Philox rounds 2-3 for h = n >> 1 (the third,
// lo(M0 h), is one multiply and is recomputed).
struct __align__(16) SiteRec {
  uint32_t jxp, jxm, jyp, jym;
  uint32_t jzp, jzm, ua, ub;
};

template <int L, int W, int NT>
struct SweepShape {
  static constexpr int N = L * L * L;
  static constexpr int ROWS = L * L;
  static constexpr int NP = NT / W;  // row partitions
  static constexpr int TJ = 4 * W;   // replicas per tile
  static constexpr size_t SPIN_BYTES = (size_t)N * W * 4;
  static constexpr size_t SMEM = SPIN_BYTES + (size_t)N * sizeof(SiteRec) + (size_t)TJ * 4;
  static_assert(NT % W == 0, "threads must tile the words of a row");
  static_assert(32 % W == 0, "a warp must cover whole rows");
};

// Interleave the L/2 Philox blocks of a row round by round (1), or leave the
// schedule of the L/2 independent blocks to the compiler (0).
#ifndef PA_SWEEP_ROUND_MAJOR
#define PA_SWEEP_ROUND_MAJOR 1
#endif
// 64-bit products as one wide multiply (0) or as separate high/low multiplies (1).
#ifndef PA_SWEEP_SPLIT_MUL
#define PA_SWEEP_SPLIT_MUL 0
#endif

__device__ __forceinline__ void mulhilo(uint32_t m, uint32_t a, uint32_t& hi, uint32_t& lo) {
#if PA_SWEEP_SPLIT_MUL
  asm("mul.hi.u32 %0, %1, %2;" : "=r"(hi) : "r"(m), "r"(a));
  asm("mul.lo.u32 %0, %1, %2;" : "=r"(lo) : "r"(m), "r"(a));
#else
  hi = __umulhi(m, a);
  lo = m * a;
#endif
}

// Rows are visited in parity-class order: rho < L^2/2 are the rows with
// (y + z) even, the rest odd, so consecutive rows share the x-offset of their
// colour-c sites (a warp spanning several rows then runs one code path).
template <int L>
__device__ __forceinline__ void row_of(int rho, int& y, int& z, int& p) {
  constexpr int HALF = L * L / 2, H = L / 2;
  p = rho >= HALF;
  const int i = rho - p * HALF;
  z = i / H;
  y = 2 * (i % H) + ((p + z) & 1);
}

// Per-thread, per-half-sweep part of rounds 1-3.
struct ThreadPhilox {
  uint32_t ta;   // lo(M1 g): XORed with the site's ua to give round-2 word 0
  uint32_t tb;   // hi(M0 A1) ^ k1_2: XORed with the site's uc to give round-2 word 2
  uint32_t tdk;  // lo(M0 A1) ^ k1_3: round-3 word 2 is hi(M0 A2) ^ tdk
};

__device__ __forceinline__ ThreadPhilox thread_philox(uint32_t g, uint32_t q, const uint32_t* k0,
                                                      const uint32_t* k1) {
  uint32_t h1, l1;
  mulhilo(kM1, g, h1, l1);
  const uint32_t a1 = h1 ^ q ^ k0[0];
  uint32_t ha, la;
  mulhilo(kM0, a1, ha, la);
  ThreadPhilox tp;
  tp.ta = l1;
  tp.tb = ha ^ k1[1];
  tp.tdk = la ^ k1[2];
  return tp;
}

// Rounds 3..10 from the hoisted parts; returns the four output words.
__device__ __forceinline__ uint4 philox_tail(const SiteRec& sr, uint32_t uc, const ThreadPhilox& tp,
                                             const uint32_t* k0, const uint32_t* k1) {
  const uint32_t a2 = sr.ua ^ tp.ta;
  const uint32_t c2 = tp.tb ^ uc;
  uint32_t h, l, h2, l2;
  mulhilo(kM1, c2, h, l);   // round 3
  mulhilo(kM0, a2, h2, l2);
  uint32_t x0 = h ^ sr.ub, x1 = l, x2 = h2 ^ tp.tdk, x3 = l2;
#pragma unroll
  for (int r = 3; r < 10; ++r) {  // rounds 4..10 (key index r)
    mulhilo(kM1, x2, h, l);
    mulhilo(kM0, x0, h2, l2);
    const uint32_t n0 = h ^ x1 ^ k0[r];
    const uint32_t n2 = h2 ^ x3 ^ k1[r];
    x0 = n0;
    x1 = l;
    x2 = n2;
    x3 = l2;
  }
  return make_uint4(x0, x1, x2, x3);
}

// Metropolis thresholds by 4u (bytes 0, 4, 8 -> u = 0, 1, 2; 12..28 unused), at a
// fixed shared-memory address so that a lookup is one load at the byte offset.
__shared__ __align__(16) uint32_t g_thr_tab[8];

// Philox blocks of the L/2 colour sites of one row.  Word b of block xh is the
// random number of replica 4g + b at site h = h0 + xh (both colours of a site
// pair share h; the half-sweep is folded into tp).  philox_init runs round 3
// from the hoisted parts; philox_rounds runs rounds [r0, r1) of all blocks.
template <int L>
__device__ __forceinline__ void philox_init(uint32_t h0, const SiteRec* __restrict__ rec, const ThreadPhilox& tp,
                                            uint32_t (&q)[4][L / 2]) {
#pragma unroll
  for (int xh = 0; xh < L / 2; ++xh) {
    const SiteRec& sr = rec[2 * xh];
    const uint32_t uc = kM0 * (h0 + (uint32_t)xh);  // lo(M0 h)
    uint32_t h, l, h2, l2;
    mulhilo(kM1, tp.tb ^ uc, h, l);
    mulhilo(kM0, sr.ua ^ tp.ta, h2, l2);
    q[0][xh] = h ^ sr.ub;
    q[1][xh] = l;
    q[2][xh] = h2 ^ tp.tdk;
    q[3][xh] = l2;
  }
}

template <int L, int R0, int R1>
__device__ __forceinline__ void philox_rounds(const uint32_t* k0, const uint32_t* k1, uint32_t (&q)[4][L / 2]) {
#pragma unroll
  for (int rr = R0; rr < R1; ++rr) {  // key index rr = round rr + 1
#pragma unroll
    for (int xh = 0; xh < L / 2; ++xh) {
      uint32_t h, l, h2, l2;
      mulhilo(kM1, q[2][xh], h, l);
      mulhilo(kM0, q[0][xh], h2, l2);
      const uint32_t n0 = h ^ q[1][xh] ^ k0[rr];
      const uint32_t n2 = h2 ^ q[3][xh] ^ k1[rr];
      q[0][xh] = n0;
      q[1][xh] = l;
      q[2][xh] = n2;
      q[3][xh] = l2;
    }
  }
}

// Rounds of the next row's Philox advanced after the update of site xh of the
// current row: rounds 4..10 (key indices 3..9) spread over the L/2 sites.
template <int L, int XH>
__device__ __forceinline__ void philox_slice(const uint32_t* k0, const uint32_t* k1, uint32_t (&q)[4][L / 2]) {
  constexpr int H = L / 2;
  constexpr int R0 = 3 + (7 * XH) / H;
  constexpr int R1 = 3 + (7 * (XH + 1)) / H;
  philox_rounds<L, R0, R1>(k0, k1, q);
}

// Metropolis update of the colour-X0 sites x = X0, X0 + 2, ... of one row from
// the row's random words q.  The row is read in full first (own row: all L
// sites, whose other-colour half are the x neighbours; the four neighbour rows:
// the L/2 sites next to the updated ones), then updated and written back.  All
// neighbour offsets are compile-time; pointers are at (row base, word).
template <int L, int W, int X0, bool NEXT>
__device__ __forceinline__ void update_row(uint32_t* __restrict__ p0, const uint32_t* __restrict__ pyp,
                                           const uint32_t* __restrict__ pym, const uint32_t* __restrict__ pzp,
                                           const uint32_t* __restrict__ pzm, const SiteRec* __restrict__ rec,
                                           const uint32_t (&q)[4][L / 2], const uint32_t* k0, const uint32_t* k1,
                                           uint32_t (&qn)[4][L / 2]) {
  constexpr int H = L / 2;
  const char* tb = reinterpret_cast<const char*>(g_thr_tab);
  uint32_t row[L], nyp[H], nym[H], nzp[H], nzm[H];
#pragma unroll
  for (int x = 0; x < L; ++x) row[x] = p0[x * W];
#pragma unroll
  for (int xh = 0; xh < H; ++xh) {
    const int x = 2 * xh + X0;
    nyp[xh] = pyp[x * W];
    nym[xh] = pym[x * W];
    nzp[xh] = pzp[x * W];
    nzm[xh] = pzm[x * W];
  }
  // phase 1: 4u per byte (unsatisfied bonds) of every site of the row
  uint32_t u4[H];
#pragma unroll
  for (int xh = 0; xh < H; ++xh) {
    const int x = 2 * xh + X0;
    const int xp = x == L - 1 ? 0 : x + 1;
    const int xm = x == 0 ? L - 1 : x - 1;
    const SiteRec& sr = rec[x];
    const uint32_t s0 = row[x];
    u4[xh] = (s0 ^ row[xp] ^ sr.jxp) + (s0 ^ row[xm] ^ sr.jxm) + (s0 ^ nyp[xh] ^ sr.jyp) + (s0 ^ nym[xh] ^ sr.jym) +
             (s0 ^ nzp[xh] ^ sr.jzp) + (s0 ^ nzm[xh] ^ sr.jzm);
  }
  // phase 2: thresholds thr(u) of every replica of the row (all loads in flight together)
  uint32_t th[4][H];
#pragma unroll
  for (int xh = 0; xh < H; ++xh) {
    th[0][xh] = *reinterpret_cast<const uint32_t*>(tb + (u4[xh] & 0xFFu));
    th[1][xh] = *reinterpret_cast<const uint32_t*>(tb + __byte_perm(u4[xh], 0u, 0x4441));
    th[2][xh] = *reinterpret_cast<const uint32_t*>(tb + __byte_perm(u4[xh], 0u, 0x4442));
    th[3][xh] = *reinterpret_cast<const uint32_t*>(tb + (u4[xh] >> 24));
  }
  // phase 3: flips and write-back
#pragma unroll
  for (int xh = 0; xh < H; ++xh) {
    const int x = 2 * xh + X0;
    uint32_t acc = row[x];  // spin bits, flipped where r < thr(u)
    if (q[0][xh] < th[0][xh]) acc ^= 0x00000004u;
    if (q[1][xh] < th[1][xh]) acc ^= 0x00000400u;
    if (q[2][xh] < th[2][xh]) acc ^= 0x00040000u;
    if (q[3][xh] < th[3][xh]) acc ^= 0x04000000u;
    // u >= 3 (dE <= 0) always flips: u4 + 0x74 reaches bit 7 exactly when u4 >= 12;
    // the table entries of those bytes are 0, so no compare above flipped them
    p0[x * W] = (acc ^ ((u4[xh] + 0x74747474u) >> 5)) & kSpinBit;
    if (NEXT) {
      if (xh == 0) philox_slice<L, 0>(k0, k1, qn);
      if (xh == 1) philox_slice<L, 1>(k0, k1, qn);
      if (xh == 2) philox_slice<L, 2>(k0, k1, qn);
      if (xh == 3) philox_slice<L, 3>(k0, k1, qn);
      if (xh == 4) philox_slice<L, 4>(k0, k1, qn);
      if (xh == 5) philox_slice<L, 5>(k0, k1, qn);
      if (xh == 6) philox_slice<L, 6>(k0, k1, qn);
      if (xh == 7) philox_slice<L, 7>(k0, k1, qn);
    }
  }
}

// Row k of a partition: rows of one parity class, interleaved across the
// partitions of that class.
template <int L, int NP>
__device__ __forceinline__ int row_index(int part, int k, int p) {
  constexpr int HALF = L * L / 2, H = L / 2, PC = NP / 2;
  const int i = (part % PC) + k * PC;  // index within the class
  const int z = i / H;
  const int y = 2 * (i % H) + ((p + z) & 1);
  return y + L * z;
  (void)HALF;
}

// All rows of one partition for one half-sweep, colour sites at x = X0 mod 2:
// the random words of row k+1 are computed in the same straight-line code as
// the update of row k, so multiply-heavy and bitwise work overlap.
template <int L, int W, int NP, int X0>
__device__ __forceinline__ void sweep_rows(uint32_t* sp, const SiteRec* recs, int part, int p, const ThreadPhilox& tp,
                                           const uint32_t* k0, const uint32_t* k1) {
  constexpr int RPP = L * L / NP;  // rows per partition
  static_assert(L / 2 <= 8, "the interleaved Philox slices cover at most 8 sites per row");
  uint32_t qa[4][L / 2], qb[4][L / 2];
  {
    const int r = row_index<L, NP>(part, 0, p);
    philox_init<L>((uint32_t)(r * L) >> 1, recs + r * L, tp, qa);
    philox_rounds<L, 3, 10>(k0, k1, qa);
  }
#pragma unroll
  for (int k = 0; k < RPP; ++k) {
    const int r = row_index<L, NP>(part, k, p);
    uint32_t(&cur)[4][L / 2] = (k & 1) ? qb : qa;
    uint32_t(&nxt)[4][L / 2] = (k & 1) ? qa : qb;
    if (k + 1 < RPP) {
      const int rn = row_index<L, NP>(part, k + 1, p);
      philox_init<L>((uint32_t)(rn * L) >> 1, recs + rn * L, tp, nxt);
    }
    const int y = r % L, z = r / L;
    const int yp = y == L - 1 ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    const int zp = z == L - 1 ? 0 : z + 1, zm = z == 0 ? L - 1 : z - 1;
    uint32_t* p0 = sp + (size_t)r * L * W;
    const uint32_t* pyp = sp + (size_t)(yp + L * z) * L * W;
    const uint32_t* pym = sp + (size_t)(ym + L * z) * L * W;
    const uint32_t* pzp = sp + (size_t)(y + L * zp) * L * W;
    const uint32_t* pzm = sp + (size_t)(y + L * zm) * L * W;
    if (k + 1 < RPP)
      update_row<L, W, X0, true>(p0, pyp, pym, pzp, pzm, recs + r * L, cur, k0, k1, nxt);
    else
      update_row<L, W, X0, false>(p0, pyp, pym, pzp, pzm, recs + r * L, cur, k0, k1, nxt);
  }
}

template <int L, int W, int NT>
__global__ void __launch_bounds__(NT) k_sweep(const __grid_constant__ SweepArgs a) {
  using S = SweepShape<L, W, NT>;
  constexpr int N = S::N, NP = S::NP, TJ = S::TJ, ROWS = S::ROWS;
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* sp = sm;                                                  // spins [N][W]
  SiteRec* recs = reinterpret_cast<SiteRec*>(sm + (size_t)N * W);     // [N]
  uint32_t* thr_tab = g_thr_tab;
  int* ecnt = reinterpret_cast<int*>(recs + N);                       // [TJ]

  const PopDev& P = a.pop;
  const uint32_t* k0 = a.k0;
  const uint32_t* k1 = a.k1;
  const int R_new = P.rec[a.t].R_tilde;
  const int tile0 = blockIdx.x * TJ;
  if (tile0 >= R_new) return;
  const int tid = threadIdx.x;
  const int word = tid % W;
  const int part = tid / W;

  // site records: bond masks and the site/step parts of Philox rounds 1-3
  for (int n = tid; n < N; n += NT) {
    const int x = n % L, y = (n / L) % L, z = n / (L * L);
    const int nxm = (x == 0 ? L - 1 : x - 1) + L * (y + L * z);
    const int nym = x + L * ((y == 0 ? L - 1 : y - 1) + L * z);
    const int nzm = x + L * (y + L * (z == 0 ? L - 1 : z - 1));
    SiteRec r;
    r.jxp = a.jtab[4 * n + 0] & kSpinBit;
    r.jyp = a.jtab[4 * n + 1] & kSpinBit;
    r.jzp = a.jtab[4 * n + 2] & kSpinBit;
    r.jxm = a.jtab[4 * nxm + 0] & kSpinBit;
    r.jym = a.jtab[4 * nym + 1] & kSpinBit;
    r.jzm = a.jtab[4 * nzm + 2] & kSpinBit;
    const uint32_t h = (uint32_t)n >> 1;
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(kM0, h, hi0, lo0);
    const uint32_t c1 = hi0 ^ (uint32_t)a.t ^ k1[0];
    mulhilo(kM1, c1, hi1, lo1);
    r.ua = hi1 ^ k0[1];
    r.ub = lo1 ^ k0[2];
    recs[n] = r;
  }
  if (tid < 8) thr_tab[tid] = tid == 0 ? a.thr12 : tid == 1 ? a.thr8 : tid == 2 ? a.thr4 : 0u;
  for (int i = tid; i < TJ; i += NT) ecnt[i] = 0;

  // 1. gather from the parents (spin bit only)
  int par[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = tile0 + 4 * word + b;
    par[b] = j < R_new ? P.parents[j] : -1;
  }
  const int8_t* src = P.spins[a.cur];
  // four consecutive, word-aligned parents: one 32-bit load per site
  const bool contiguous = par[0] >= 0 && (par[0] & 3) == 0 && par[1] == par[0] + 1 && par[2] == par[0] + 2 &&
                          par[3] == par[0] + 3;
  // Rows are gathered GB at a time with every load issued before the first
  // use, so each thread keeps 4 GB independent loads in flight.
  constexpr int GB = (N / NP) % 10 == 0 ? 10 : ((N / NP) % 8 == 0 ? 8 : ((N / NP) % 4 == 0 ? 4 : 1));
  for (int n0 = part; n0 < N; n0 += NP * GB) {
    uint32_t v[GB][4];
#pragma unroll
    for (int i = 0; i < GB; ++i) {
      const int n = n0 + i * NP;
      const int8_t* row = src + (size_t)(n < N ? n : 0) * a.pitch;
      if (contiguous) {
        v[i][0] = *reinterpret_cast<const uint32_t*>(row + par[0]);
      } else {
#pragma unroll
        for (int b = 0; b < 4; ++b) v[i][b] = par[b] >= 0 ? (uint32_t)(uint8_t)row[par[b]] : 0x01u;
      }
    }
#pragma unroll
    for (int i = 0; i < GB; ++i) {
      const int n = n0 + i * NP;
      const uint32_t w = contiguous ? v[i][0] : (v[i][0] | (v[i][1] << 8) | (v[i][2] << 16) | (v[i][3] << 24));
      if (n < N) sp[n * W + word] = w & kSpinBit;
    }
  }
  __syncthreads();

  // 2. sweeps: partition `part` owns rows of parity class p = (y + z) & 1; in
  // half-sweep c its colour sites sit at x = p ^ c mod 2 in every row.
  static_assert(NP % 2 == 0 && (ROWS / 2) % (NP / 2) == 0, "row partitions must split each parity class");
  const uint32_t g = (uint32_t)(tile0 >> 2) + (uint32_t)word;
  const int pclass = part / (NP / 2);
  uint32_t* spw = sp + word;
  for (int s = 0; s < a.n_sweeps; ++s) {
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const ThreadPhilox tp = thread_philox(g, 2u * (uint32_t)s + (uint32_t)c, k0, k1);
      if ((pclass ^ c) == 0)
        sweep_rows<L, W, NP, 0>(spw, recs, part, pclass, tp, k0, k1);
      else
        sweep_rows<L, W, NP, 1>(spw, recs, part, pclass, tp, k0, k1);
      __syncthreads();
    }
  }

  // 3. energy levels: unsatisfied forward bonds of every site (4 per bond per byte)
  {
    int cnt[4] = {0, 0, 0, 0};
    for (int r = part; r < ROWS; r += NP) {
      const int y = r % L, z = r / L;
      const int yp = y == L - 1 ? 0 : y + 1, zp = z == L - 1 ? 0 : z + 1;
      const uint32_t* p0 = sp + (size_t)r * L * W + word;
      const uint32_t* pyp = sp + (size_t)(yp + L * z) * L * W + word;
      const uint32_t* pzp = sp + (size_t)(y + L * zp) * L * W + word;
      const SiteRec* rr = recs + r * L;
      uint32_t acc = 0;  // <= 12 L per byte
#pragma unroll
      for (int x = 0; x < L; ++x) {
        const int xp = x == L - 1 ? 0 : x + 1;
        const uint32_t s0 = p0[x * W];
        acc += (s0 ^ p0[xp * W] ^ rr[x].jxp) + (s0 ^ pyp[x * W] ^ rr[x].jyp) + (s0 ^ pzp[x * W] ^ rr[x].jzp);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) cnt[b] += (acc >> (8 * b)) & 0xFFu;
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) atomicAdd(&ecnt[4 * word + b], cnt[b]);
  }
  __syncthreads();
  uint32_t* hist = P.hist + (size_t)a.t * a.n_levels;
  for (int i = tid; i < TJ; i += NT) {
    const int j = tile0 + i;
    if (j < R_new) {
      const int k = ecnt[i] >> 2;
      P.levels[j] = k;
      atomicAdd(&hist[k], 1u);
    }
  }

  // 4. store the tile as int8 +1 (0x01) / -1 (0xFF)
  uint32_t* dst = reinterpret_cast<uint32_t*>(P.spins[1 - a.cur]);
  const int64_t pw = a.pitch / 4;
  for (int n = part; n < N; n += NP) dst[n * pw + (tile0 >> 2) + word] = (sp[n * W + word] >> 2) * 0xFEu + 0x01010101u;
}

template <int L, int W, int NT>
static int launch_t(const RunGeom& g, const SweepArgs& args, cudaStream_t s) {
  using S = SweepShape<L, W, NT>;
  cudaError_t e = cudaFuncSetAttribute(k_sweep<L, W, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
  if (e != cudaSuccess) return (int)e;
  dim3 grid((unsigned)((g.R_cap + S::TJ - 1) / S::TJ));
  k_sweep<L, W, NT><<<grid, NT, S::SMEM, s>>>(args);
  return (int)cudaGetLastError();
}

bool sweep_supported(int L) { return L >= 2 && L <= kMaxL && L % 2 == 0; }

int launch_sweep(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, int t, int n_sweeps,
                 const uint32_t met_thr[3], void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < g.n_pop; ++i) {
    SweepArgs args;
    args.pop = pops[i];
    uint32_t k0 = pops[i].key_met[0], k1 = pops[i].key_met[1];
    for (int r = 0; r < 10; ++r) {
      args.k0[r] = k0;
      args.k1[r] = k1;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    args.jtab = jtab;
    args.pitch = g.pitch;
    args.n_levels = g.n_levels;
    args.t = t;
    args.cur = cur;
    args.n_sweeps = n_sweeps;
    args.thr4 = met_thr[0];
    args.thr8 = met_thr[1];
    args.thr12 = met_thr[2];
    int e;
    switch (g.L) {
      case 2: e = launch_t<2, 32, 128>(g, args, s); break;
      case 4: e = launch_t<4, 32, 256>(g, args, s); break;
      case 6: e = launch_t<6, 32, 384>(g, args, s); break;
      case 8: e = launch_t<8, 32, 512>(g, args, s); break;
      case 10: e = launch_t<10, PA_SWEEP_W_L10, PA_SWEEP_NT_L10>(g, args, s); break;
      case 12: e = launch_t<12, 16, 576>(g, args, s); break;
      case 14: e = launch_t<14, 8, 224>(g, args, s); break;
      case 16: e = launch_t<16, 4, 256>(g, args, s); break;
      default: e = (int)cudaErrorInvalidValue;
    }
    if (e != 0) return e;
  }
  return 0;
}

}  // namespace pa
