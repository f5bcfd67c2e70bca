// pa_sweep.cu — the Metropolis sweep kernel (the dominant cost of a PA step).
//
// One CTA owns a tile of TJ = 8W consecutive slots of the NEW population and
// all N sites of those replicas in shared memory (W 32-bit words per site row,
// eight replicas per word, one 4-bit nibble each).  It
//   1. gathers each slot's spins from its parent in the old population (the
//      replica copy of the resampling, §II, fused into the load),
//   2. runs S checkerboard Metropolis sweeps at beta_t in shared memory (colour
//      c = (x + y + z) & 1, colour 0 then colour 1; the neighbours of a site all
//      have the other colour, so all sites of one colour update independently),
//   3. counts each replica's unsatisfied bonds (its energy level k) and adds
//      the tile to the level histogram of step t, and
//   4. writes the tile to the new population buffer (int8 +1 / -1).
// HBM traffic is one read and one write of the tile per step, whatever S is.
//
// Metropolis rule: flipping s_n costs dE = 2 s_n h_n = 12 - 4u, u = unsatisfied
// bonds at n.  It is taken when u >= 3 (dE <= 0), or with probability
// thr / 2^32, thr = floor(2^32 exp(-beta dE)), read as a 32-bit uniform in two
// halves: the replica's 16-bit uniform U against the top half of thr decides
// unless the two are equal (probability 2^-16), and only then the tie-break
// uniform V against the low half.  U is half (j & 1) of word (j & 7) >> 1 of
// Philox4x32-10 at counter (n >> 1, 2s + c, j >> 3, t) keyed by (run_seed,
// Metropolis, population): one block serves the eight replicas of a word.  V is
// the same half of the same word under the tie-break key.
//
// Shared-memory encoding: replica i of a word is nibble i, spin -1 <=> bit 0
// set.  For a bond, s_a ^ s_b ^ Jmask (Jmask = 1 per nibble for J = -1) is 1
// exactly when the bond is unsatisfied, so the nibble-wise sum of the six bond
// terms plus 5 is v = u + 5 in [5, 11]: bit 3 of v says u >= 3 (always flip),
// and a byte of v (replicas 2k and 2k+1) indexes a 256-entry table holding both
// replicas' thresholds, so one 64-bit shared load serves the two replicas whose
// uniforms share Philox word k.  Comparing that whole word with a threshold
// decides the high-half replica whenever it is not tied, and the low half
// shifted up decides the other; a tie anywhere in a site sends it to tie_corrections,
// which recomputes both blocks and corrects the tied replicas.
//
// Philox hoisting (same function, fewer multiplies): with counter words
// (h, q, g, t) = (site, half-sweep, group, step), the round-1 and round-2
// products depend either on the site and step only (tabulated once per launch
// in shared memory) or on the thread and half-sweep only (registers), so each
// block costs the 16 wide multiplies of rounds 3..10, two per update.
#include <cuda_runtime.h>

#include "pa_device.cuh"
#include "pa_internal.h"

// Build-time knobs of the sweep's launch shape and code generation.
#ifndef PA_SWEEP_ROW_UNROLL
#define PA_SWEEP_ROW_UNROLL 8  // rows of a partition unrolled per loop trip (8: all of them)
#endif

namespace pa {

constexpr int kSweepRowUnroll = PA_SWEEP_ROW_UNROLL;
constexpr uint32_t kM0 = 0xD2511F53u;
constexpr uint32_t kM1 = 0xCD9E8D57u;
constexpr uint32_t kNib = 0x11111111u;   // bit 0 of every nibble: the spin bit
constexpr uint32_t kBias = 0x55555555u;  // 5 per nibble

struct SweepArgs {
  PopDev pop;
  const uint32_t* jtab;  // [N][4] forward-bond masks (non-zero for J = -1)
  int64_t pitch;
  int32_t n_levels;
  int32_t t;
  int32_t cur;
  int32_t n_sweeps;
  uint32_t thr4, thr8, thr12;
  uint32_t k0[10];  // Metropolis round keys of this population
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
  static constexpr int TJ = 8 * W;   // replicas per tile
  static constexpr size_t SMEM = (size_t)N * W * 4 + (size_t)N * sizeof(SiteRec) + (size_t)TJ * 4;
  static_assert(NT % W == 0, "threads must tile the words of a row");
  static_assert(32 % W == 0, "a warp must cover whole rows");
  static_assert(L % 2 == 0 && L / 2 <= 8, "even L up to 16");
  static_assert(NP % 2 == 0 && (ROWS / 2) % (NP / 2) == 0, "row partitions must split each parity class");
};

// Thresholds of two replicas by one byte of v = u + 5 (low nibble: .x, high
// nibble: .y); entries for u >= 3 are 0 (those flips come from bit 3 of v).
__shared__ __align__(16) uint2 g_thr_pair[256];

__device__ __forceinline__ void mulhilo(uint32_t m, uint32_t a, uint32_t& hi, uint32_t& lo) {
  hi = __umulhi(m, a);
  lo = m * a;
}

// Per-thread, per-half-sweep part of rounds 1-3 of one group g.
struct ThreadPhilox {
  uint32_t ta;   // lo(M1 g): XORed with the site's ua to give round-2 word 0
  uint32_t tb;   // hi(M0 A1) ^ k1_2: XORed with lo(M0 h) to give round-2 word 2
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

// Philox blocks (rounds 3..10) of one colour site h for the two groups of a
// word: w8[b] is word b of group 0's block (b < 4) or group 1's (b >= 4).
__device__ __forceinline__ void philox_site(uint32_t h, const SiteRec& sr, const ThreadPhilox& tpa,
                                            const ThreadPhilox& tpb, const uint32_t* k0, const uint32_t* k1,
                                            uint32_t (&w8)[8]) {
  const uint32_t uc = kM0 * h;  // lo(M0 h)
#pragma unroll
  for (int gi = 0; gi < 2; ++gi) {
    const ThreadPhilox& tp = gi ? tpb : tpa;
    uint32_t hh, l, h2, l2;
    mulhilo(kM1, tp.tb ^ uc, hh, l);
    mulhilo(kM0, sr.ua ^ tp.ta, h2, l2);
    w8[4 * gi + 0] = hh ^ sr.ub;
    w8[4 * gi + 1] = l;
    w8[4 * gi + 2] = h2 ^ tp.tdk;
    w8[4 * gi + 3] = l2;
  }
#pragma unroll
  for (int rr = 3; rr < 10; ++rr) {
#pragma unroll
    for (int gi = 0; gi < 2; ++gi) {
      uint32_t hh, l, h2, l2;
      mulhilo(kM1, w8[4 * gi + 2], hh, l);
      mulhilo(kM0, w8[4 * gi + 0], h2, l2);
      const uint32_t n0 = hh ^ w8[4 * gi + 1] ^ k0[rr];
      const uint32_t n2 = h2 ^ w8[4 * gi + 3] ^ k1[rr];
      w8[4 * gi + 0] = n0;
      w8[4 * gi + 1] = l;
      w8[4 * gi + 2] = n2;
      w8[4 * gi + 3] = l2;
    }
  }
}

// Philox blocks (rounds 3..10) of the L/2 colour sites of one row for the one
// group of a word (+-1 couplings): q[b][xh] is word b at site h = h0 + xh.
template <int L>
__device__ __forceinline__ void philox_row1(uint32_t h0, const SiteRec* __restrict__ rec, const ThreadPhilox& tp,
                                            const uint32_t* k0, const uint32_t* k1, uint32_t (&q)[4][L / 2]) {
  constexpr int H = L / 2;
#pragma unroll
  for (int xh = 0; xh < H; ++xh) {  // round 3 from the hoisted parts
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
#pragma unroll
  for (int rr = 3; rr < 10; ++rr) {  // rounds 4..10 (key index rr)
#pragma unroll
    for (int xh = 0; xh < H; ++xh) {
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

// Full Philox4x32-10 block from the per-round keys k0[r], k1[r].
__device__ __forceinline__ void philox_rounds(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t* k0,
                                              const uint32_t* k1, uint32_t (&o)[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t h0, l0, h1, l1;
    mulhilo(kM0, c0, h0, l0);
    mulhilo(kM1, c2, h1, l1);
    c0 = h1 ^ c1 ^ k0[r];
    c1 = l1;
    c2 = h0 ^ c3 ^ k1[r];
    c3 = l0;
  }
  o[0] = c0;
  o[1] = c1;
  o[2] = c2;
  o[3] = c3;
}

// Corrections for the tied replicas of one word at one site (v = u + 5 per
// nibble, counter (h, qc, g, t)): bit 4i is set where replica i's exact decision
// (the tie-break uniform against the low half of its threshold) differs from the
// one the fast test took.  Rare, so both blocks are recomputed.
// Its inputs are plain values and key pointers: handing it the kernel's argument
// block instead made the fast path of the sweep about 5% slower on GB300.
__device__ __noinline__ uint32_t tie_corrections(uint32_t v, uint32_t h, uint32_t qc, uint32_t g, uint32_t t,
                                                 const uint32_t* k0, const uint32_t* k1, const uint32_t* ktie) {
  const char* tb = reinterpret_cast<const char*>(g_thr_pair);
  uint32_t om[4];
  philox_rounds(h, qc, g, t, k0, k1, om);
  const uint4 otv = philox4x32_10(make_uint4(h, qc, g, t), ktie[0], ktie[1]);
  const uint32_t ot[4] = {otv.x, otv.y, otv.z, otv.w};
  uint32_t corr = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint2 th = *reinterpret_cast<const uint2*>(tb + (((v >> (8 * k)) & 0xFFu) << 3));
    const uint32_t r = om[k], rl = r << 16;
    if (((rl ^ th.x) < 0x10000u) && ((rl < th.x) != ((ot[k] & 0xFFFFu) < (th.x & 0xFFFFu)))) corr ^= 1u << (8 * k);
    if (((r ^ th.y) < 0x10000u) && ((r < th.y) != ((ot[k] >> 16) < (th.y & 0xFFFFu)))) corr ^= 1u << (8 * k + 4);
  }
  return corr;
}

// Metropolis update of the colour sites x = X0, X0 + 2, ... of one row from the
// row's random words q (counter words h0 + xh, qc, g).  The row is read in full
// first (own row: all L sites, whose other-colour half are the x neighbours;
// the four neighbour rows: the L/2 sites next to the updated ones).  All
// neighbour offsets are compile-time; pointers are at (row base, this thread's word).
template <int L, int W, int X0>
__device__ __forceinline__ void update_row(uint32_t* __restrict__ p0, const uint32_t* __restrict__ pyp,
                                           const uint32_t* __restrict__ pym, const uint32_t* __restrict__ pzp,
                                           const uint32_t* __restrict__ pzm, const SiteRec* __restrict__ rec,
                                           const uint32_t (&q)[4][L / 2], uint32_t h0, uint32_t qc, uint32_t g,
                                           uint32_t t, const uint32_t* k0, const uint32_t* k1, const uint32_t* ktie) {
  constexpr int H = L / 2;
  const char* tb = reinterpret_cast<const char*>(g_thr_pair);
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
  // v = u + 5 per nibble, u = unsatisfied bonds of each replica at the site
  uint32_t v[H];
#pragma unroll
  for (int xh = 0; xh < H; ++xh) {
    const int x = 2 * xh + X0;
    const int xp = x == L - 1 ? 0 : x + 1;
    const int xm = x == 0 ? L - 1 : x - 1;
    const SiteRec& sr = rec[x];
    const uint32_t s0 = row[x];
    v[xh] = (s0 ^ row[xp] ^ sr.jxp) + (s0 ^ row[xm] ^ sr.jxm) + (s0 ^ nyp[xh] ^ sr.jyp) + (s0 ^ nym[xh] ^ sr.jym) +
            (s0 ^ nzp[xh] ^ sr.jzp) + (s0 ^ nzm[xh] ^ sr.jzm) + kBias;
  }
  // flips: replicas 2k and 2k+1 (byte k of v) read the low and high halves of word k
  uint32_t acc[H];
  uint32_t tied = 0;  // bit xh: some replica of site xh has its uniform equal to its threshold's top half
#pragma unroll
  for (int xh = 0; xh < H; ++xh) {
    const int x = 2 * xh + X0;
    uint32_t f = row[x];
    bool tie = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint2 th = *reinterpret_cast<const uint2*>(tb + (k == 0 ? ((v[xh] << 3) & 0x7F8u)
                                                                     : ((v[xh] >> (8 * k - 3)) & 0x7F8u)));
      const uint32_t r = q[k][xh];
      const uint32_t rl = r << 16;
      if (rl < th.x) f ^= 1u << (8 * k);
      if (r < th.y) f ^= 1u << (8 * k + 4);
      tie = tie || ((rl ^ th.x) < 0x10000u) || ((r ^ th.y) < 0x10000u);
    }
    acc[xh] = f;
    if (tie) tied |= 1u << xh;
  }
  if (tied) {
#pragma unroll
    for (int xh = 0; xh < H; ++xh)
      if ((tied >> xh) & 1u) acc[xh] ^= tie_corrections(v[xh], h0 + (uint32_t)xh, qc, g, t, k0, k1, ktie);
  }
#pragma unroll
  for (int xh = 0; xh < H; ++xh) {
    const int x = 2 * xh + X0;
    p0[x * W] = (acc[xh] ^ (v[xh] >> 3)) & kNib;  // bit 3 of v: u >= 3 always flips
  }
}

// Row k of a partition: rows of one parity class (y + z) & 1 = p, interleaved
// across the partitions of that class.
template <int L, int NP>
__device__ __forceinline__ int row_index(int part, int k, int p) {
  constexpr int H = L / 2, PC = NP / 2;
  const int i = (part % PC) + k * PC;  // index within the class
  const int z = i / H;
  const int y = 2 * (i % H) + ((p + z) & 1);
  return y + L * z;
}

// All rows of one partition for one half-sweep; the colour sites sit at
// x = X0 mod 2 in every row of the partition's parity class.
template <int L, int W, int NP, int X0>
__device__ __forceinline__ void sweep_rows(uint32_t* sp, const SiteRec* recs, int part, int p, const ThreadPhilox& tp,
                                           const uint32_t* k0, const uint32_t* k1, uint32_t qc, uint32_t g, uint32_t t,
                                           const uint32_t* ktie) {
  constexpr int RPP = L * L / NP;  // rows per partition
  constexpr int UNROLL = RPP < kSweepRowUnroll ? RPP : kSweepRowUnroll;
#pragma unroll UNROLL
  for (int k = 0; k < RPP; ++k) {
    const int r = row_index<L, NP>(part, k, p);
    const uint32_t h0 = (uint32_t)(r * L) >> 1;
    uint32_t q[4][L / 2];
    philox_row1<L>(h0, recs + r * L, tp, k0, k1, q);
    const int y = r % L, z = r / L;
    const int yp = y == L - 1 ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    const int zp = z == L - 1 ? 0 : z + 1, zm = z == 0 ? L - 1 : z - 1;
    update_row<L, W, X0>(sp + (size_t)r * L * W, sp + (size_t)(yp + L * z) * L * W, sp + (size_t)(ym + L * z) * L * W,
                         sp + (size_t)(y + L * zp) * L * W, sp + (size_t)(y + L * zm) * L * W, recs + r * L, q, h0,
                         qc, g, t, k0, k1, ktie);
  }
}

// int8 spins (0x01 / 0xFF) of four replicas -> nibbles 0..3 (bit 1 of a byte is the sign)
__device__ __forceinline__ uint32_t bytes_to_nibbles(uint32_t w) {
  const uint32_t b = (w >> 1) & 0x01010101u;
  return (b & 1u) | ((b >> 4) & 0x10u) | ((b >> 8) & 0x100u) | ((b >> 12) & 0x1000u);
}
// nibbles 0..3 of x -> four int8 spins
__device__ __forceinline__ uint32_t nibbles_to_bytes(uint32_t x) {
  const uint32_t b = (x & 1u) | ((x & 0x10u) << 4) | ((x & 0x100u) << 8) | ((x & 0x1000u) << 12);
  return b * 0xFEu + 0x01010101u;
}

// ---- phases of a tile shared by both sweep kernels (nt consumer threads take part)

// Site records (bond masks, site/step parts of Philox rounds 1-3) and the
// threshold-pair table; all `nthreads` threads of the CTA help.
template <int L>
__device__ __forceinline__ void init_tables(const SweepArgs& a, SiteRec* recs, int tid, int nthreads) {
  constexpr int N = L * L * L;
  const uint32_t* k0 = a.k0;
  const uint32_t* k1 = a.k1;
  for (int n = tid; n < N; n += nthreads) {
    const int x = n % L, y = (n / L) % L, z = n / (L * L);
    const int nxm = (x == 0 ? L - 1 : x - 1) + L * (y + L * z);
    const int nym = x + L * ((y == 0 ? L - 1 : y - 1) + L * z);
    const int nzm = x + L * (y + L * (z == 0 ? L - 1 : z - 1));
    SiteRec r;
    r.jxp = a.jtab[4 * n + 0] ? kNib : 0u;
    r.jyp = a.jtab[4 * n + 1] ? kNib : 0u;
    r.jzp = a.jtab[4 * n + 2] ? kNib : 0u;
    r.jxm = a.jtab[4 * nxm + 0] ? kNib : 0u;
    r.jym = a.jtab[4 * nym + 1] ? kNib : 0u;
    r.jzm = a.jtab[4 * nzm + 2] ? kNib : 0u;
    const uint32_t h = (uint32_t)n >> 1;
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(kM0, h, hi0, lo0);
    const uint32_t c1 = hi0 ^ (uint32_t)a.t ^ k1[0];
    mulhilo(kM1, c1, hi1, lo1);
    r.ua = hi1 ^ k0[1];
    r.ub = lo1 ^ k0[2];
    recs[n] = r;
  }
  for (int b = tid; b < 256; b += nthreads) {
    const int lo = (b & 15) - 5, hi = (b >> 4) - 5;  // u of the two replicas
    const uint32_t tlo = lo == 0 ? a.thr12 : lo == 1 ? a.thr8 : lo == 2 ? a.thr4 : 0u;
    const uint32_t thi = hi == 0 ? a.thr12 : hi == 1 ? a.thr8 : hi == 2 ? a.thr4 : 0u;
    g_thr_pair[b] = make_uint2(tlo, thi);
  }
}

// Gather the tile's spins from the parents of its slots (nibble-packed).
template <int L, int W, int NP>
__device__ __forceinline__ void gather_tile(const SweepArgs& a, uint32_t* sp, int tile0, int R_new, int word,
                                            int part) {
  constexpr int N = L * L * L;
  const PopDev& P = a.pop;
  int par[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int j = tile0 + 8 * word + b;
    par[b] = j < R_new ? P.parents[j] : -1;
  }
  bool contiguous = par[0] >= 0 && (par[0] & 7) == 0;
#pragma unroll
  for (int b = 1; b < 8; ++b) contiguous = contiguous && par[b] == par[0] + b;
  const int8_t* src = P.spins[a.cur];
  // rows are gathered GB at a time with every load issued before the first use
  constexpr int GB = (N / NP) % 10 == 0 ? 10 : ((N / NP) % 8 == 0 ? 8 : ((N / NP) % 4 == 0 ? 4 : 1));
  for (int n0 = part; n0 < N; n0 += NP * GB) {
    uint2 vv[GB];
#pragma unroll
    for (int i = 0; i < GB; ++i) {
      const int n = n0 + i * NP;
      const int8_t* row = src + (size_t)(n < N ? n : 0) * a.pitch;
      if (contiguous) {
        vv[i] = *reinterpret_cast<const uint2*>(row + par[0]);
      } else {
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          lo |= (par[b] >= 0 ? (uint32_t)(uint8_t)row[par[b]] : 0x01u) << (8 * b);
          hi |= (par[b + 4] >= 0 ? (uint32_t)(uint8_t)row[par[b + 4]] : 0x01u) << (8 * b);
        }
        vv[i] = make_uint2(lo, hi);
      }
    }
#pragma unroll
    for (int i = 0; i < GB; ++i) {
      const int n = n0 + i * NP;
      if (n < N) sp[n * W + word] = bytes_to_nibbles(vv[i].x) | (bytes_to_nibbles(vv[i].y) << 16);
    }
  }
}

// Unsatisfied forward bonds of every replica of the tile, summed into ecnt.
template <int L, int W, int NP>
__device__ __forceinline__ void count_levels(const uint32_t* sp, const SiteRec* recs, int* ecnt, int word, int part) {
  constexpr int ROWS = L * L;
  int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int r = part; r < ROWS; r += NP) {
    const int y = r % L, z = r / L;
    const int yp = y == L - 1 ? 0 : y + 1, zp = z == L - 1 ? 0 : z + 1;
    const uint32_t* p0 = sp + (size_t)r * L * W + word;
    const uint32_t* pyp = sp + (size_t)(yp + L * z) * L * W + word;
    const uint32_t* pzp = sp + (size_t)(y + L * zp) * L * W + word;
    const SiteRec* rr = recs + r * L;
    uint32_t even = 0, odd = 0;  // nibbles 0,2,4,6 / 1,3,5,7 in byte lanes, <= 3L each
#pragma unroll
    for (int x = 0; x < L; ++x) {
      const int xp = x == L - 1 ? 0 : x + 1;
      const uint32_t s0 = p0[x * W];
      const uint32_t e = (s0 ^ p0[xp * W] ^ rr[x].jxp) + (s0 ^ pyp[x * W] ^ rr[x].jyp) + (s0 ^ pzp[x * W] ^ rr[x].jzp);
      even += e & 0x0F0F0F0Fu;
      odd += (e >> 4) & 0x0F0F0F0Fu;
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      cnt[2 * b] += (even >> (8 * b)) & 0xFFu;
      cnt[2 * b + 1] += (odd >> (8 * b)) & 0xFFu;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) atomicAdd(&ecnt[8 * word + i], cnt[i]);
}

// Levels and histogram of the tile's slots (after count_levels and a barrier).
template <int TJ>
__device__ __forceinline__ void publish_levels(const SweepArgs& a, const int* ecnt, int tile0, int R_new, int tid,
                                               int nthreads) {
  const PopDev& P = a.pop;
  uint32_t* hist = P.hist + (size_t)a.t * a.n_levels;
  for (int i = tid; i < TJ; i += nthreads) {
    const int j = tile0 + i;
    if (j < R_new) {
      const int k = ecnt[i];
      P.levels[j] = k;
      atomicAdd(&hist[k], 1u);
    }
  }
}

// Write the tile back as int8 +1 (0x01) / -1 (0xFF).
template <int L, int W, int NP>
__device__ __forceinline__ void store_tile(const SweepArgs& a, const uint32_t* sp, int tile0, int word, int part) {
  constexpr int N = L * L * L;
  int8_t* dst = a.pop.spins[1 - a.cur];
  for (int n = part; n < N; n += NP) {
    const uint32_t w = sp[n * W + word];
    *reinterpret_cast<uint2*>(dst + (size_t)n * a.pitch + tile0 + 8 * word) =
        make_uint2(nibbles_to_bytes(w), nibbles_to_bytes(w >> 16));
  }
}

// Row-partitioned sweep kernel: every warp generates its own random words and
// updates its rows.
template <int L, int W, int NT, int MB>
__global__ void __launch_bounds__(NT, MB) k_sweep(const __grid_constant__ SweepArgs a) {
  using S = SweepShape<L, W, NT>;
  constexpr int N = S::N, NP = S::NP, TJ = S::TJ;
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* sp = sm;                                               // spins [N][W]
  SiteRec* recs = reinterpret_cast<SiteRec*>(sm + (size_t)N * W);  // [N]
  int* ecnt = reinterpret_cast<int*>(recs + N);                    // [TJ]
  const int R_new = a.pop.rec[a.t].R_tilde;
  const int tile0 = blockIdx.x * TJ;
  if (tile0 >= R_new) return;
  const int tid = threadIdx.x, word = tid % W, part = tid / W;
  init_tables<L>(a, recs, tid, NT);
  for (int i = tid; i < TJ; i += NT) ecnt[i] = 0;
  gather_tile<L, W, NP>(a, sp, tile0, R_new, word, part);
  __syncthreads();

  // sweeps: partition `part` owns rows of parity class p = (y + z) & 1; in
  // half-sweep c its colour sites sit at x = p ^ c mod 2 in every row.
  const uint32_t g = (uint32_t)(tile0 >> 3) + (uint32_t)word;  // Philox group: the word's eight replicas
  const int pclass = part / (NP / 2);
  uint32_t* spw = sp + word;
  for (int s = 0; s < a.n_sweeps; ++s) {
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const uint32_t q = 2u * (uint32_t)s + (uint32_t)c;
      const ThreadPhilox tp = thread_philox(g, q, a.k0, a.k1);
      if ((pclass ^ c) == 0)
        sweep_rows<L, W, NP, 0>(spw, recs, part, pclass, tp, a.k0, a.k1, q, g, (uint32_t)a.t, a.pop.key_tie);
      else
        sweep_rows<L, W, NP, 1>(spw, recs, part, pclass, tp, a.k0, a.k1, q, g, (uint32_t)a.t, a.pop.key_tie);
      __syncthreads();
    }
  }
  count_levels<L, W, NP>(sp, recs, ecnt, word, part);
  __syncthreads();
  publish_levels<TJ>(a, ecnt, tile0, R_new, tid, NT);
  store_tile<L, W, NP>(a, sp, tile0, word, part);
}

// ---- Gaussian couplings (§II.A): the same tiles, gather, store and Philox words;
// the acceptance of a flip comes from per-site tables built on the host for the
// step's beta.  For each half of a site's bonds (x+1, x-1, y+1 | y-1, z+1, z-1)
// and each pattern of antiparallel neighbours (bit k: bond k of the half), the
// table holds that half's energy change dE_h (fixed point, units of 2^-20) and
// F_h = (float) exp(-beta dE_h).  A flip is taken when dE_1 + dE_2 <= 0, or
// when the Philox word is below min(floor(2^32 F_1 F_2), 2^32 - 1) with the
// product rounded once in FP32.  Energies are recounted from scratch after the
// sweeps: E = -sum J + 2 sum over antiparallel bonds of J (exact integers).

struct GSweepArgs {
  SweepArgs base;
  const GTabEntry* gtab;  // [N][2][8] acceptance tables of this step
  const int32_t* Jq;      // [3N] fixed-point couplings of the forward bonds
  long long Jtot;         // sum of all couplings
};

template <int L, int W, int NP, int X0>
__device__ __forceinline__ void sweep_rows_g(uint32_t* sp, const SiteRec* recs, int part, int p,
                                             const ThreadPhilox& tpa, const ThreadPhilox& tpb, const uint32_t* k0,
                                             const uint32_t* k1, const GTabEntry* __restrict__ gtab) {
  constexpr int H = L / 2, RPP = L * L / NP;
  const int2* tab = reinterpret_cast<const int2*>(gtab);
#pragma unroll 1
  for (int k = 0; k < RPP; ++k) {
    const int r = row_index<L, NP>(part, k, p);
    const int y = r % L, z = r / L;
    const int yp = y == L - 1 ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    const int zp = z == L - 1 ? 0 : z + 1, zm = z == 0 ? L - 1 : z - 1;
    uint32_t* p0 = sp + (size_t)r * L * W;
    const uint32_t* pyp = sp + (size_t)(yp + L * z) * L * W;
    const uint32_t* pym = sp + (size_t)(ym + L * z) * L * W;
    const uint32_t* pzp = sp + (size_t)(y + L * zp) * L * W;
    const uint32_t* pzm = sp + (size_t)(y + L * zm) * L * W;
    uint32_t row[L];
#pragma unroll
    for (int x = 0; x < L; ++x) row[x] = p0[x * W];
#pragma unroll
    for (int xh = 0; xh < H; ++xh) {
      const int x = 2 * xh + X0;
      const int xp = x == L - 1 ? 0 : x + 1;
      const int xm = x == 0 ? L - 1 : x - 1;
      uint32_t w8[8];
      philox_site((uint32_t)(r * L) / 2u + (uint32_t)xh, recs[r * L + x], tpa, tpb, k0, k1, w8);
      const uint32_t s0 = row[x];
      const uint32_t P1 = (s0 ^ row[xp]) | ((s0 ^ row[xm]) << 1) | ((s0 ^ pyp[x * W]) << 2);
      const uint32_t P2 = (s0 ^ pym[x * W]) | ((s0 ^ pzp[x * W]) << 1) | ((s0 ^ pzm[x * W]) << 2);
      const int2* tb = tab + (size_t)(r * L + x) * 16;
      uint32_t flip = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int2 e1 = __ldg(tb + ((P1 >> (4 * i)) & 7u));
        const int2 e2 = __ldg(tb + 8 + ((P2 >> (4 * i)) & 7u));
        const float pr = __fmul_rn(__int_as_float(e1.y), __int_as_float(e2.y));
        const uint32_t thr = __float2uint_rz(__fmul_rn(pr, 4294967296.0f));
        if (e1.x + e2.x <= 0 || w8[i] < thr) flip |= 1u << (4 * i);
      }
      p0[x * W] = s0 ^ flip;
    }
  }
}

// Antiparallel forward bonds of every replica of the tile weighted by J, summed into ecnt.
template <int L, int W, int NP>
__device__ __forceinline__ void count_energies_g(const uint32_t* sp, const int32_t* __restrict__ Jq, long long* ecnt,
                                                 int word, int part) {
  constexpr int ROWS = L * L;
  int acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // |sum| < 2^31 for every launch shape in use
  for (int r = part; r < ROWS; r += NP) {
    const int y = r % L, z = r / L;
    const int yp = y == L - 1 ? 0 : y + 1, zp = z == L - 1 ? 0 : z + 1;
    const uint32_t* p0 = sp + (size_t)r * L * W + word;
    const uint32_t* pyp = sp + (size_t)(yp + L * z) * L * W + word;
    const uint32_t* pzp = sp + (size_t)(y + L * zp) * L * W + word;
#pragma unroll
    for (int x = 0; x < L; ++x) {
      const int xp = x == L - 1 ? 0 : x + 1;
      const int n = r * L + x;
      const uint32_t s0 = p0[x * W];
      const uint32_t ax = s0 ^ p0[xp * W], ay = s0 ^ pyp[x * W], az = s0 ^ pzp[x * W];
      const int jx = __ldg(Jq + 3 * n), jy = __ldg(Jq + 3 * n + 1), jz = __ldg(Jq + 3 * n + 2);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        acc[i] += (jx & -(int)((ax >> (4 * i)) & 1u)) + (jy & -(int)((ay >> (4 * i)) & 1u)) +
                  (jz & -(int)((az >> (4 * i)) & 1u));
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
    atomicAdd(reinterpret_cast<unsigned long long*>(&ecnt[8 * word + i]), (unsigned long long)(long long)acc[i]);
}

template <int L, int W, int NT, int MB>
__global__ void __launch_bounds__(NT, MB) k_sweep_g(const __grid_constant__ GSweepArgs ga) {
  using S = SweepShape<L, W, NT>;
  constexpr int N = S::N, NP = S::NP, TJ = S::TJ;
  const SweepArgs& a = ga.base;
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* sp = sm;
  SiteRec* recs = reinterpret_cast<SiteRec*>(sm + (size_t)N * W);
  long long* ecnt = reinterpret_cast<long long*>(recs + N);
  const int R_new = a.pop.rec[a.t].R_tilde;
  const int tile0 = blockIdx.x * TJ;
  if (tile0 >= R_new) return;
  const int tid = threadIdx.x, word = tid % W, part = tid / W;
  init_tables<L>(a, recs, tid, NT);
  for (int i = tid; i < TJ; i += NT) ecnt[i] = 0;
  gather_tile<L, W, NP>(a, sp, tile0, R_new, word, part);
  __syncthreads();
  const uint32_t g0 = 2u * ((uint32_t)(tile0 >> 3) + (uint32_t)word);
  const int pclass = part / (NP / 2);
  uint32_t* spw = sp + word;
  for (int s = 0; s < a.n_sweeps; ++s) {
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const uint32_t q = 2u * (uint32_t)s + (uint32_t)c;
      const ThreadPhilox tpa = thread_philox(g0, q, a.k0, a.k1);
      const ThreadPhilox tpb = thread_philox(g0 + 1u, q, a.k0, a.k1);
      if ((pclass ^ c) == 0)
        sweep_rows_g<L, W, NP, 0>(spw, recs, part, pclass, tpa, tpb, a.k0, a.k1, ga.gtab);
      else
        sweep_rows_g<L, W, NP, 1>(spw, recs, part, pclass, tpa, tpb, a.k0, a.k1, ga.gtab);
      __syncthreads();
    }
  }
  count_energies_g<L, W, NP>(sp, ga.Jq, ecnt, word, part);
  __syncthreads();
  for (int i = tid; i < TJ; i += NT) {
    const int j = tile0 + i;
    if (j < R_new) a.pop.E64[j] = -ga.Jtot + 2 * ecnt[i];
  }
  store_tile<L, W, NP>(a, sp, tile0, word, part);
}

template <int L, int W, int NT, int MB>
static int launch_g_t(const RunGeom& g, const GSweepArgs& args, cudaStream_t s) {
  using S = SweepShape<L, W, NT>;
  const size_t smem = S::SMEM + (size_t)S::TJ * 4;  // energy counters are 8 bytes, not 4
  cudaError_t e = cudaFuncSetAttribute(k_sweep_g<L, W, NT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  dim3 grid((unsigned)((g.R_cap + S::TJ - 1) / S::TJ));
  k_sweep_g<L, W, NT, MB><<<grid, NT, smem, s>>>(args);
  return (int)cudaGetLastError();
}

template <int L, int W, int NT, int MB>
static int launch_t(const RunGeom& g, const SweepArgs& args, cudaStream_t s) {
  using S = SweepShape<L, W, NT>;
  cudaError_t e =
      cudaFuncSetAttribute(k_sweep<L, W, NT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
  if (e != cudaSuccess) return (int)e;
  dim3 grid((unsigned)((g.R_cap + S::TJ - 1) / S::TJ));
  k_sweep<L, W, NT, MB><<<grid, NT, S::SMEM, s>>>(args);
  return (int)cudaGetLastError();
}

namespace {

// Candidate launch shapes: words per site row W (8W replicas per tile),
// threads per CTA, CTAs per SM the kernel is compiled for (its register cap).
// The first entry of each L is the default (the fastest measured on GB300);
// the autotuner may pick another.  All give identical results.  At L = 14 no
// shape with whole warps keeps 8W | 256 and fits: 784 and 392 threads leave a
// partial last warp and one warp whose rows straddle the two parity classes
// (it runs both colour offsets; still far faster than 224 threads).
struct ShapeEntry {
  int L, W, NT, MB;
  size_t smem;
  int (*launch)(const RunGeom&, const SweepArgs&, cudaStream_t);
};
#define PA_SHAPE(L, W, NT, MB) {L, W, NT, MB, SweepShape<L, W, NT>::SMEM, &launch_t<L, W, NT, MB>}
const ShapeEntry kShapes[] = {
    PA_SHAPE(2, 32, 128, 1),
    PA_SHAPE(4, 32, 256, 3),   PA_SHAPE(4, 32, 256, 1),  PA_SHAPE(4, 32, 512, 2),
    PA_SHAPE(6, 32, 384, 2),   PA_SHAPE(6, 32, 384, 1),  PA_SHAPE(6, 32, 576, 1),
    PA_SHAPE(8, 32, 512, 2),   PA_SHAPE(8, 32, 512, 1),  PA_SHAPE(8, 32, 256, 2),
    PA_SHAPE(10, 32, 640, 1),  PA_SHAPE(10, 16, 320, 2),
    PA_SHAPE(12, 16, 768, 1),  PA_SHAPE(12, 16, 576, 1), PA_SHAPE(12, 8, 384, 2),
    PA_SHAPE(14, 8, 784, 1),   PA_SHAPE(14, 4, 392, 1),
    PA_SHAPE(16, 4, 512, 1),   PA_SHAPE(16, 4, 1024, 1),
};
#undef PA_SHAPE
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

const ShapeEntry* shape_of(int L, int i) {
  if (i < 0) return nullptr;
  for (int k = 0; k < kNumShapes; ++k)
    if (kShapes[k].L == L && i-- == 0) return &kShapes[k];
  return nullptr;
}

}  // namespace

bool sweep_supported(int L) { return L >= 2 && L <= kMaxL && L % 2 == 0; }

int sweep_shape_count(int L) {
  int n = 0;
  for (int k = 0; k < kNumShapes; ++k) n += kShapes[k].L == L;
  return n;
}

bool sweep_shape_info(int L, int i, SweepShapeInfo* out) {
  const ShapeEntry* e = shape_of(L, i);
  if (!e || !out) return false;
  out->L = e->L;
  out->W = e->W;
  out->NT = e->NT;
  out->MB = e->MB;
  out->smem = (int32_t)e->smem;
  return true;
}

int launch_sweep(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, int t, int n_sweeps,
                 const uint32_t met_thr[3], void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const ShapeEntry* shape = shape_of(g.L, g.sweep_shape);
  if (!shape) return (int)cudaErrorInvalidValue;
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
    const int e = shape->launch(g, args, s);
    if (e != 0) return e;
  }
  return 0;
}

int launch_g_sweep(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, const int32_t* Jq, long long Jtot,
                   const GTabEntry* gtab, int t, int n_sweeps, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < g.n_pop; ++i) {
    GSweepArgs ga;
    SweepArgs& args = ga.base;
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
    args.thr4 = args.thr8 = args.thr12 = 0u;
    ga.gtab = gtab;
    ga.Jq = Jq;
    ga.Jtot = Jtot;
    int e;
    switch (g.L) {  // one launch shape per L, compiled for one CTA per SM (no register spills)
      case 2: e = launch_g_t<2, 32, 128, 1>(g, ga, s); break;
      case 4: e = launch_g_t<4, 32, 256, 1>(g, ga, s); break;
      case 6: e = launch_g_t<6, 32, 384, 1>(g, ga, s); break;
      case 8: e = launch_g_t<8, 32, 512, 1>(g, ga, s); break;
      case 10: e = launch_g_t<10, 32, 640, 1>(g, ga, s); break;
      case 12: e = launch_g_t<12, 16, 576, 1>(g, ga, s); break;
      case 14: e = launch_g_t<14, 8, 784, 1>(g, ga, s); break;
      case 16: e = launch_g_t<16, 4, 512, 1>(g, ga, s); break;
      default: e = (int)cudaErrorInvalidValue;
    }
    if (e != 0) return e;
  }
  return 0;
}

}  // namespace pa
