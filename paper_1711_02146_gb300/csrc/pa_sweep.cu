// pa_sweep.cu — the Metropolis sweep kernels (the dominant cost of a PA step).
//
// One CTA owns a tile of consecutive slots of the NEW population and all N sites
// of those replicas in shared memory.  It
//   1. gathers each slot's spins from its parent in the old population (the
//      replica copy of the resampling, §II, fused into the load),
//   2. runs S checkerboard Metropolis sweeps at beta_t in shared memory (colour
//      c = (x + y + z) & 1, colour 0 then colour 1; the neighbours of a site all
//      have the other colour, so all sites of one colour update independently),
//   3. counts each replica's energy and adds the tile to the histogram of step t,
//   4. writes the tile to the new population buffer (int8 +1 / -1),
//   5. (+-1 couplings) adds the families of its slots to the step's family
//      statistics (§III.A), so the step needs no family launch of its own.
// HBM traffic is one read and one write of the tile per step, whatever S is.
//
// +-1 couplings (k_sweep): bit-sliced tiles.  Word w of a site row holds slots
// tile0 + 32w + b as bit b (set for spin -1), so one 32-bit logic instruction
// tests a bond, adds a bit or takes a comparison step for 32 replicas.  Flipping
// s_n costs dE = 12 - 4u, u = unsatisfied bonds at n; u comes from the six
// bond bits by a tree of full adders as three bit planes.  u >= 3 (dE <= 0)
// always flips; otherwise the flip is taken when the replica's 32-bit uniform r
// is below thr(u) = floor(2^32 exp(-beta dE)).  r is the replica's bit column:
// bit 31 - p of r is bit b of word p mod 4 of Philox4x32-10 at counter
// (n >> 1, 2s + c, 8 (slot >> 5) + p / 4, t) keyed by (run_seed, Metropolis,
// population), so one block gives four bit planes of 32 replicas' uniforms.
// A replica is decided at the first plane, from the top, where its bit differs
// from its threshold's (accepted if the threshold has the 1): two planes on
// average.  Blocks 0 and 1 (planes 0..7) are always drawn and compared as one
// 8-bit bit-sliced subtraction (its borrow is "below", plus an "equal so far"
// mask); the words with replicas still equal draw further blocks on demand.
//
// Philox hoisting (same function, fewer multiplies): with counter words
// (h, q, g, t) = (site, half-sweep, group, step), the round-1 and round-2
// products depend either on the site and step only (tabulated once per launch
// in shared memory) or on the thread and half-sweep only (registers), so each
// block costs the 16 wide multiplies of rounds 3..10.
//
// Gaussian couplings (k_sweep_g, below): nibble-packed tiles, eight replicas per
// word, with one Philox block per site for a word's eight replicas (the upper 16
// bits of their uniforms; the lower 16 bits only on a tie).
#include <cuda_runtime.h>

#include <algorithm>

#include "pa_device.cuh"
#include "pa_family.cuh"
#include "pa_internal.h"

namespace pa {

constexpr uint32_t kM0 = 0xD2511F53u;
constexpr uint32_t kM1 = 0xCD9E8D57u;

struct SweepArgs {
  PopDev pop;
  const uint32_t* jtab;  // [N][4] forward-bond masks (non-zero for J = -1)
  int64_t pitch;
  int32_t n_levels;
  int32_t t;
  int32_t cur;
  int32_t n_sweeps;
  int32_t slot_base;  // global slot of local slot 0 (Philox groups are global); 0 for a whole population
  int32_t fam;        // 1: add the tile's families to the step record (not for one rank's share)
  // this launch's first local slot (tile 0 of the grid), and the split of a two-launch
  // sweep: slots below `split` in tiles of tj_main, the rest in tiles of tj_tail
  int32_t tile_base, split, tj_main, tj_tail;
  uint32_t thr4, thr8, thr12;
  uint32_t k0[10];  // Metropolis round keys of this population
  uint32_t k1[10];
  // +-1: plane p's threshold bit as a function of the unsatisfied-bond count u
  // (bits u0, u1; u = 0, 1, 2): T(u) = bit 31 - p of thr(u) as an all-zero / all-one
  // word, stored as tm[p] = {T(0), T(0) ^ T(1), T(0) ^ T(2)}, so that the bit of a
  // replica is tm[p][0] ^ (u0 & tm[p][1]) ^ (u1 & tm[p][2]) (u >= 3 never compares)
  uint32_t tm[32][4];
  uint32_t live[4];    // +-1: the same form of "thr(u) > 0" (a replica with thr(u) = 0 never flips)
};

// Per-site shared-memory record: the six bond masks of the site (all ones for
// J = -1), and the site/step-dependent parts of Philox rounds 2-3 for h = n >> 1
// (the third, lo(M0 h), is one multiply and is recomputed).
struct __align__(16) SiteRec {
  uint32_t jxp, jxm, jyp, jym;
  uint32_t jzp, jzm, ua, ub;
};

// Nibble tiles of the Gaussian kernel: 8 replicas per word.
template <int L, int W, int NT>
struct SweepShape {
  static constexpr int N = L * L * L;
  static constexpr int ROWS = L * L;
  static constexpr int NP = NT / W;  // row partitions
  static constexpr int TJ = 8 * W;   // replicas per tile
  static constexpr int RPP = ROWS / NP;  // rows per partition
  static constexpr size_t SMEM = (size_t)N * W * 4 + (size_t)N * sizeof(SiteRec) + (size_t)TJ * 4;
  static constexpr size_t SMEM_ROWS = (size_t)NP * RPP * 8 * sizeof(int);  // the row table
  static_assert(NT % W == 0, "threads must tile the words of a row");
  static_assert(32 % W == 0, "a warp must cover whole rows");
  static_assert(L % 2 == 0 && L / 2 <= 8, "even L up to 16");
  static_assert(NP % 2 == 0 && (ROWS / 2) % (NP / 2) == 0, "row partitions must split each parity class");
};

// 32 x 32 -> 64-bit product as one wide multiply (2.4 % faster sweep than the
// separate high and low products).
__device__ __forceinline__ void mulhilo(uint32_t m, uint32_t a, uint32_t& hi, uint32_t& lo) {
  uint64_t p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(m));
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
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

// Per partition and row (rows of the partition's parity class, row_index), the
// word offsets of the row and of its four neighbour rows in a tile of W words per
// site and the row's first site: {row, y+1, y-1, z+1, first site, z-1}.  A
// thread's rows never change, so each tile fills this once.
template <int L, int W, int NP>
__device__ __forceinline__ void fill_row_table(int* rowtab, int tid, int nthreads) {
  constexpr int RPP = L * L / NP;
  for (int e = tid; e < NP * RPP; e += nthreads) {
    const int pt = e / RPP, kr = e % RPP;
    const int r = row_index<L, NP>(pt, kr, pt / (NP / 2));
    const int y = r % L, z = r / L;
    const int yp = y == L - 1 ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    const int zp = z == L - 1 ? 0 : z + 1, zm = z == 0 ? L - 1 : z - 1;
    int* o = rowtab + 8 * e;
    o[0] = r * L * W;
    o[1] = (yp + L * z) * L * W;
    o[2] = (ym + L * z) * L * W;
    o[3] = (y + L * zp) * L * W;
    o[4] = r * L;
    o[5] = (y + L * zm) * L * W;
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

// ---- phases of a tile: init_tables and publish_levels serve both kernels,
// gather_tile and store_tile are the Gaussian kernel's (nibble tiles)

// Site records (bond masks, site/step parts of Philox rounds 1-3); all
// `nthreads` threads of the CTA help.
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
    r.jxp = a.jtab[4 * n + 0] ? ~0u : 0u;
    r.jyp = a.jtab[4 * n + 1] ? ~0u : 0u;
    r.jzp = a.jtab[4 * n + 2] ? ~0u : 0u;
    r.jxm = a.jtab[4 * nxm + 0] ? ~0u : 0u;
    r.jym = a.jtab[4 * nym + 1] ? ~0u : 0u;
    r.jzm = a.jtab[4 * nzm + 2] ? ~0u : 0u;
    const uint32_t h = (uint32_t)n >> 1;
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(kM0, h, hi0, lo0);
    const uint32_t c1 = hi0 ^ (uint32_t)a.t ^ k1[0];
    mulhilo(kM1, c1, hi1, lo1);
    r.ua = hi1 ^ k0[1];
    r.ub = lo1 ^ k0[2];
    recs[n] = r;
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

// ---- +-1 couplings: the bit-sliced sweep

// Bits needed to hold 0..n.
constexpr int bits_for(int n) { return n < 2 ? 1 : 1 + bits_for(n / 2); }

// A word whose replicas the first two Philox blocks (bit planes 0..7) leave
// undecided: its site n and word (n | word << 16), the undecided replicas, and
// bits 0 and 1 of their unsatisfied-bond counts.
struct __align__(16) Deferred {
  uint32_t loc, eq, u0, u1;
};
constexpr int kQueueCap = 64;  // a warp queues at most 31 + 32 words before it finishes 32 of them

template <int L, int W, int NT, int MB>
struct BitShape {
  static constexpr int N = L * L * L;
  static constexpr int ROWS = L * L;
  static constexpr int NP = NT / W;       // row partitions
  static constexpr int TJ = 32 * W;       // replicas per tile
  static constexpr int SLOTS = 33 * W;    // parents (padded by one per word), then level counts
  static constexpr int CB = bits_for(3 * L * (ROWS / NP));  // bit planes of a thread's level counter
  static constexpr size_t SMEM_TILE = (size_t)N * W * 4 + (size_t)N * sizeof(SiteRec) + (size_t)SLOTS * 4;
  static constexpr size_t SMEM_QUEUES = (size_t)(NT / 32) * kQueueCap * sizeof(Deferred);
  static constexpr int RPP = ROWS / NP;  // rows per partition
  static constexpr size_t SMEM_ROWS = (size_t)NP * RPP * 8 * sizeof(int);
  // Deferred comparisons need whole warps that each stay inside one parity class
  // (every lane of a warp then runs the same half-sweep code in step), and room
  // for the queues without fewer than MB CTAs per SM (228 KB per SM, 1 KB of it
  // reserved per CTA).
  static constexpr bool DEFER = NT % 32 == 0 && ((NP / 2) * W) % 32 == 0 &&
                                (size_t)MB * (SMEM_TILE + SMEM_QUEUES + SMEM_ROWS + 1024) <= 233472;
  static constexpr int NQ = DEFER ? NT / 32 : 0;  // one queue per warp
  static constexpr size_t SMEM = SMEM_TILE + (DEFER ? SMEM_QUEUES + SMEM_ROWS : 0);
  static_assert(NT % W == 0 && 32 % W == 0 && NT <= 1024, "threads must tile the words of a row");
  static_assert(L % 2 == 0 && L / 2 <= 8, "even L up to 16");
  static_assert(NP % 2 == 0 && (ROWS / 2) % (NP / 2) == 0, "row partitions must split each parity class");
  static_assert(1024 % TJ == 0, "a tile never crosses the 1024-slot pitch unit");
};

__device__ __forceinline__ uint32_t majority(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (c & (a ^ b)); }

// One Philox block (rounds 3..10 from the hoisted parts) of site h, uc = lo(M0 h),
// for the thread's group of block index b (its ThreadPhilox tp).
__device__ __forceinline__ void philox_block(uint32_t uc, const SiteRec& sr, const ThreadPhilox& tp, const uint32_t* k0,
                                             const uint32_t* k1, uint32_t (&w)[4]) {
  uint32_t hh, l, h2, l2;
  mulhilo(kM1, tp.tb ^ uc, hh, l);
  mulhilo(kM0, sr.ua ^ tp.ta, h2, l2);
  w[0] = hh ^ sr.ub;
  w[1] = l;
  w[2] = h2 ^ tp.tdk;
  w[3] = l2;
#pragma unroll
  for (int rr = 3; rr < 10; ++rr) {  // rounds 4..10 (key index rr)
    mulhilo(kM1, w[2], hh, l);
    mulhilo(kM0, w[0], h2, l2);
    const uint32_t n0 = hh ^ w[1] ^ k0[rr];
    const uint32_t n2 = h2 ^ w[3] ^ k1[rr];
    w[0] = n0;
    w[1] = l;
    w[2] = n2;
    w[3] = l2;
  }
}

// The plane's threshold bit of each replica of a word (SweepArgs::tm), from bits
// u0, u1 of its unsatisfied-bond count.
__device__ __forceinline__ uint32_t threshold_bits(const uint32_t* tm, uint32_t u0, uint32_t u1) {
  return tm[0] ^ (u0 & tm[1]) ^ (u1 & tm[2]);
}

// One plane of the comparison uniform < threshold for the 32 replicas of a word,
// most significant plane first: r holds the plane's bit of every replica's
// uniform.  eq: replicas whose uniform has matched its threshold so far; acc:
// replicas decided below it.
__device__ __forceinline__ void compare_plane(uint32_t r, uint32_t u0, uint32_t u1, const uint32_t* tm, uint32_t& eq,
                                              uint32_t& acc) {
  const uint32_t t = threshold_bits(tm, u0, u1);
  acc |= eq & t & ~r;
  eq &= ~(r ^ t);
}

// One plane of the same comparison taken least significant plane first, as the
// borrow of a bit-sliced subtraction r - thr: after the planes p..7, lt holds the
// replicas whose bits p..7 of r are below those of thr, same those whose bits
// p..7 are equal.
__device__ __forceinline__ void borrow_plane(uint32_t r, uint32_t u0, uint32_t u1, const uint32_t* tm, uint32_t& lt,
                                             uint32_t& same) {
  const uint32_t t = threshold_bits(tm, u0, u1);
  lt = (~r & t) | (~(r ^ t) & lt);
  same &= ~(r ^ t);
}

// One half-sweep of the rows of partition `part` (parity class p, colour sites at
// x = X0 mod 2).  spw points at this thread's word of site 0; tp[b] are the
// thread's hoisted Philox parts of block b for this half-sweep q; g8 = 8 x the
// thread's global word index (the group of block b is g8 + b).
template <int L, int W, int NP, int X0>
__device__ __forceinline__ void sweep_rows_bits(uint32_t* spw, const SiteRec* recs, int part, int p,
                                                const ThreadPhilox (&tp)[4], uint32_t q, uint32_t g8,
                                                const SweepArgs& a) {
  constexpr int H = L / 2, RPP = L * L / NP;
#pragma unroll 1
  for (int k = 0; k < RPP; ++k) {
    const int r = row_index<L, NP>(part, k, p);
    const int y = r % L, z = r / L;
    const int yp = y == L - 1 ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    const int zp = z == L - 1 ? 0 : z + 1, zm = z == 0 ? L - 1 : z - 1;
    uint32_t* p0 = spw + (size_t)r * L * W;
    const uint32_t* pyp = spw + (size_t)(yp + L * z) * L * W;
    const uint32_t* pym = spw + (size_t)(ym + L * z) * L * W;
    const uint32_t* pzp = spw + (size_t)(y + L * zp) * L * W;
    const uint32_t* pzm = spw + (size_t)(y + L * zm) * L * W;
    const SiteRec* rr = recs + r * L;
    const uint32_t h0 = (uint32_t)(r * L) >> 1;
#pragma unroll 2  // two sites in flight: measured 3 % faster than one, as fast as all
    for (int xh = 0; xh < H; ++xh) {
      const int x = 2 * xh + X0;
      const int xp = x == L - 1 ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
      const SiteRec sr = rr[x];
      const uint32_t s0 = p0[x * W];
      // unsatisfied bonds (one bit per replica) and their count u in three planes
      const uint32_t b0 = s0 ^ p0[xp * W] ^ sr.jxp, b1 = s0 ^ p0[xm * W] ^ sr.jxm;
      const uint32_t b2 = s0 ^ pyp[x * W] ^ sr.jyp, b3 = s0 ^ pym[x * W] ^ sr.jym;
      const uint32_t b4 = s0 ^ pzp[x * W] ^ sr.jzp, b5 = s0 ^ pzm[x * W] ^ sr.jzm;
      const uint32_t sa = b0 ^ b1 ^ b2, ca = majority(b0, b1, b2);
      const uint32_t sb = b3 ^ b4 ^ b5, cb = majority(b3, b4, b5);
      const uint32_t u0 = sa ^ sb, k2 = sa & sb;
      const uint32_t u1 = ca ^ cb ^ k2, u2 = majority(ca, cb, k2);
      const uint32_t always = u2 | (u1 & u0);  // u >= 3: dE <= 0
      // replicas to compare: u = 0, 1, 2 (dE = 12, 8, 4) with thr(u) > 0
      uint32_t eq = ~always & threshold_bits(a.live, u0, u1);
      uint32_t acc = 0;
      const uint32_t uc = kM0 * (h0 + (uint32_t)xh);  // lo(M0 h), h = n >> 1
      {
        uint32_t w0[4], w1[4];
        philox_block(uc, sr, tp[0], a.k0, a.k1, w0);
        philox_block(uc, sr, tp[1], a.k0, a.k1, w1);
#pragma unroll
        for (int i = 0; i < 4; ++i) compare_plane(w0[i], u0, u1, a.tm[i], eq, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i) compare_plane(w1[i], u0, u1, a.tm[4 + i], eq, acc);
      }
      if (eq) {
        uint32_t w[4];
        philox_block(uc, sr, tp[2], a.k0, a.k1, w);
#pragma unroll
        for (int i = 0; i < 4; ++i) compare_plane(w[i], u0, u1, a.tm[8 + i], eq, acc);
      }
      if (eq) {
        uint32_t w[4];
        philox_block(uc, sr, tp[3], a.k0, a.k1, w);
#pragma unroll
        for (int i = 0; i < 4; ++i) compare_plane(w[i], u0, u1, a.tm[12 + i], eq, acc);
      }
#pragma unroll 1
      for (int b = 4; b < 8 && eq; ++b) {  // rare: some replica matched its threshold for 16 bits
        const ThreadPhilox tb = thread_philox(g8 + (uint32_t)b, q, a.k0, a.k1);
        uint32_t w[4];
        philox_block(uc, sr, tb, a.k0, a.k1, w);
#pragma unroll
        for (int i = 0; i < 4; ++i) compare_plane(w[i], u0, u1, a.tm[4 * b + i], eq, acc);
      }
      p0[x * W] = s0 ^ (acc | always);
    }
  }
}

// Finishes a deferred word: Philox blocks 2, 3, ... of its site and group until
// every queued replica is decided, then flips the accepted ones (the word's owner
// has already applied the flips decided in planes 0..7).  Any lane of the owner's
// warp may run it: the same-colour sites of a half-sweep are independent.
template <int W>
__device__ __forceinline__ void finish_deferred(uint32_t* sp, const SiteRec* recs, const Deferred d, uint32_t q,
                                                uint32_t gbase, const SweepArgs& a) {
  const int n = (int)(d.loc & 0xffffu), word = (int)(d.loc >> 16);
  const uint32_t u0 = d.u0, u1 = d.u1;
  uint32_t eq = d.eq, acc = 0;
  const uint32_t g8 = 8u * (gbase + (uint32_t)word);
  const uint32_t uc = kM0 * ((uint32_t)n >> 1);
  const SiteRec sr = recs[n];
#pragma unroll 1
  for (int b = 2; b < 8 && eq; ++b) {
    const ThreadPhilox tb = thread_philox(g8 + (uint32_t)b, q, a.k0, a.k1);
    uint32_t w[4];
    philox_block(uc, sr, tb, a.k0, a.k1, w);
#pragma unroll
    for (int i = 0; i < 4; ++i) compare_plane(w[i], u0, u1, a.tm[4 * b + i], eq, acc);
  }
  sp[n * W + word] ^= acc;
}

// One half-sweep of the rows of partition `part`, as sweep_rows_bits, for shapes
// whose warps stay inside one parity class: a word still undecided after blocks
// 0 and 1 (about one in eight) goes to the warp's queue dq, and whenever 32 are
// queued the warp finishes them with all lanes (finish_deferred); the rest are
// finished at the end of the half-sweep.  The decisions are the same; only the
// lanes that take them change.  sp: the tile (word-major within a site row);
// gbase: the tile's first word index (Philox group 8 (gbase + word) + b); rowtab:
// per partition and row the word offsets of the row and its four neighbour rows
// and the row's first site (built once per tile: a thread's rows never change).
// The sites of a row are unrolled, so every column offset is a constant.
template <int L, int W, int NP, int X0>
__device__ __forceinline__ void sweep_rows_bits_dq(uint32_t* sp, int word, const SiteRec* recs, int part, int p,
                                                   const ThreadPhilox (&tp)[2], uint32_t q, uint32_t gbase,
                                                   Deferred* dq, const int* rowtab, const SweepArgs& a) {
  constexpr int H = L / 2, RPP = L * L / NP;
  const int lane = (int)(threadIdx.x & 31u);
  const unsigned below = (1u << lane) - 1u;
  uint32_t* spw = sp + word;
  int head = 0, cnt = 0;  // the same in every lane of the warp
#pragma unroll 1
  for (int k = 0; k < RPP; ++k) {
    const int4 e0 = *reinterpret_cast<const int4*>(rowtab + 8 * (part * RPP + k));
    const int rL = rowtab[8 * (part * RPP + k) + 4];
    uint32_t* p0 = spw + e0.x;
    const uint32_t* pyp = spw + e0.y;
    const uint32_t* pym = spw + e0.z;
    const uint32_t* pzp = spw + e0.w;
    const uint32_t* pzm = spw + rowtab[8 * (part * RPP + k) + 5];
    const SiteRec* rr = recs + rL;
    const uint32_t h0 = (uint32_t)rL >> 1;
#pragma unroll
    for (int xh = 0; xh < H; ++xh) {
      const int x = 2 * xh + X0;
      const int xp = x == L - 1 ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
      const SiteRec sr = rr[x];
      const uint32_t s0 = p0[x * W];
      const uint32_t b0 = s0 ^ p0[xp * W] ^ sr.jxp, b1 = s0 ^ p0[xm * W] ^ sr.jxm;
      const uint32_t b2 = s0 ^ pyp[x * W] ^ sr.jyp, b3 = s0 ^ pym[x * W] ^ sr.jym;
      const uint32_t b4 = s0 ^ pzp[x * W] ^ sr.jzp, b5 = s0 ^ pzm[x * W] ^ sr.jzm;
      const uint32_t sa = b0 ^ b1 ^ b2, ca = majority(b0, b1, b2);
      const uint32_t sb = b3 ^ b4 ^ b5, cb = majority(b3, b4, b5);
      const uint32_t u0 = sa ^ sb, k2 = sa & sb;
      const uint32_t u1 = ca ^ cb ^ k2, u2 = majority(ca, cb, k2);
      const uint32_t always = u2 | (u1 & u0);  // u >= 3: dE <= 0
      // replicas to compare: u = 0, 1, 2 (dE = 12, 8, 4) with thr(u) > 0
      const uint32_t cmp = ~always & threshold_bits(a.live, u0, u1);
      uint32_t lt = 0, eq = cmp;
      const uint32_t uc = kM0 * (h0 + (uint32_t)xh);  // lo(M0 h), h = n >> 1
      {
        uint32_t w0[4], w1[4];
        philox_block(uc, sr, tp[0], a.k0, a.k1, w0);
        philox_block(uc, sr, tp[1], a.k0, a.k1, w1);
        // bits 31..24 of each uniform against those of its threshold, lowest plane first
#pragma unroll
        for (int i = 3; i >= 0; --i) borrow_plane(w1[i], u0, u1, a.tm[4 + i], lt, eq);
#pragma unroll
        for (int i = 3; i >= 0; --i) borrow_plane(w0[i], u0, u1, a.tm[i], lt, eq);
      }
      p0[x * W] = s0 ^ ((cmp & lt) | always);
      const unsigned dm = __ballot_sync(0xffffffffu, eq != 0u);
      if (eq) {
        Deferred d;
        d.loc = (uint32_t)(rL + x) | ((uint32_t)word << 16);
        d.eq = eq;
        d.u0 = u0;
        d.u1 = u1;
        dq[(head + cnt + __popc(dm & below)) & (kQueueCap - 1)] = d;
      }
      cnt += __popc(dm);
      if (cnt >= 32) {
        __syncwarp();
        finish_deferred<W>(sp, recs, dq[(head + lane) & (kQueueCap - 1)], q, gbase, a);
        __syncwarp();
        head = (head + 32) & (kQueueCap - 1);
        cnt -= 32;
      }
    }
  }
  __syncwarp();
  if (lane < cnt) finish_deferred<W>(sp, recs, dq[(head + lane) & (kQueueCap - 1)], q, gbase, a);
  __syncwarp();
}

// Gather the tile's spins from the parents of its slots into bit words; spar
// holds the tile's parents (-1 past R~), slot i at index 33 (i >> 5) + (i & 31).
template <int L, int W, int NP>
__device__ __forceinline__ void gather_bits(const SweepArgs& a, uint32_t* sp, const int* spar, int word, int part) {
  constexpr int N = L * L * L;
  int par[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) par[b] = spar[33 * word + b];
  bool contiguous = par[0] >= 0 && (par[0] & 15) == 0;
#pragma unroll
  for (int b = 1; b < 32; ++b) contiguous = contiguous && par[b] == par[0] + b;
  const int8_t* src = a.pop.spins[a.cur];
  for (int n = part; n < N; n += NP) {
    const int8_t* row = src + (size_t)n * a.pitch;
    uint32_t bits = 0;
    if (contiguous) {
      const uint4* v = reinterpret_cast<const uint4*>(row + par[0]);
      const uint4 lo = v[0], hi = v[1];
      const uint32_t q8[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)  // bit 1 of each byte is the sign; gather four of them
        bits |= ((((q8[i] >> 1) & 0x01010101u) * 0x01020408u) >> 24) << (4 * i);
    } else {
#pragma unroll
      for (int b = 0; b < 32; ++b)
        if (par[b] >= 0) bits |= (((uint32_t)(uint8_t)row[par[b]] >> 1) & 1u) << b;
    }
    sp[n * W + word] = bits;
  }
}

// Unsatisfied forward bonds of every replica of the tile, counted per thread in
// CB bit planes and then added per replica into ecnt (slot i at index i).
template <int L, int W, int NP, int CB>
__device__ __forceinline__ void count_levels_bits(const uint32_t* sp, const SiteRec* recs, int* ecnt, int word,
                                                  int part) {
  constexpr int ROWS = L * L;
  uint32_t c[CB];
#pragma unroll
  for (int i = 0; i < CB; ++i) c[i] = 0;
  for (int r = part; r < ROWS; r += NP) {
    const int y = r % L, z = r / L;
    const int yp = y == L - 1 ? 0 : y + 1, zp = z == L - 1 ? 0 : z + 1;
    const uint32_t* p0 = sp + (size_t)r * L * W + word;
    const uint32_t* pyp = sp + (size_t)(yp + L * z) * L * W + word;
    const uint32_t* pzp = sp + (size_t)(y + L * zp) * L * W + word;
    const SiteRec* rr = recs + r * L;
#pragma unroll
    for (int x = 0; x < L; ++x) {
      const int xp = x == L - 1 ? 0 : x + 1;
      const uint32_t s0 = p0[x * W];
      const uint32_t e0 = s0 ^ p0[xp * W] ^ rr[x].jxp, e1 = s0 ^ pyp[x * W] ^ rr[x].jyp,
                     e2 = s0 ^ pzp[x * W] ^ rr[x].jzp;
      const uint32_t sum = e0 ^ e1 ^ e2, two = majority(e0, e1, e2);  // e0 + e1 + e2 = sum + 2 two
      uint32_t carry = c[0] & sum;
      c[0] ^= sum;
      const uint32_t c1 = c[1] ^ two ^ carry;
      carry = majority(c[1], two, carry);
      c[1] = c1;
#pragma unroll
      for (int i = 2; i < CB; ++i) {
        const uint32_t ci = c[i] ^ carry;
        carry &= c[i];
        c[i] = ci;
      }
    }
  }
#pragma unroll 1
  for (int bb = 0; bb < 32; ++bb) {
    const int b = (bb + word) & 31;  // lanes of a warp hit different banks
    int k = 0;
#pragma unroll
    for (int i = 0; i < CB; ++i) k |= (int)((c[i] >> b) & 1u) << i;
    if (k) atomicAdd(&ecnt[32 * word + b], k);
  }
}

// Write the tile back as int8 +1 (0x01) / -1 (0xFF), 32 slots per word.
template <int L, int W, int NP>
__device__ __forceinline__ void store_bits(const SweepArgs& a, const uint32_t* sp, int tile0, int word, int part) {
  constexpr int N = L * L * L;
  int8_t* dst = a.pop.spins[1 - a.cur];
  for (int n = part; n < N; n += NP) {
    const uint32_t w = sp[n * W + word];
    uint32_t q8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {  // four bits -> bit 0 of four bytes -> 0x01 / 0xFF
      const uint32_t m = (((w >> (4 * i)) & 15u) * 0x00204081u) & 0x01010101u;
      q8[i] = m * 0xFEu + 0x01010101u;
    }
    uint4* out = reinterpret_cast<uint4*>(dst + (size_t)n * a.pitch + tile0 + 32 * word);
    out[0] = make_uint4(q8[0], q8[1], q8[2], q8[3]);
    out[1] = make_uint4(q8[4], q8[5], q8[6], q8[7]);
  }
}

// Families (a7) of the tile's new slots, so that a step needs no family launch
// of its own: a family is a run of equal labels along the slots (labels ascend).
// sh (shared memory, free by now) holds labs[0..TJ] (the slot before the tile,
// then the tile's slots; -1 past R~), a bit mask per 32 slots of the slots that
// start a run, and 64 words for the final sum.  The thread at a run's first slot
// takes its end from the next start in the tile, or, for the tile's last run, by
// galloping through the labels after the tile (run_end), and records the family
// (pa_family.cuh); the last tile to finish adds the entropy.
template <int TJ, int NT>
__device__ __forceinline__ void tile_families(const SweepArgs& a, int* sh, int tile0, int R_new, int tid) {
  constexpr int NC = TJ / 32;  // chunks of 32 slots (TJ <= 1024)
  static_assert(NT % 32 == 0 || TJ <= NT, "the lanes of a warp take whole chunks");
  int* labs = sh;
  unsigned* bm = reinterpret_cast<unsigned*>(sh + TJ + 1);  // [NC + 1]: start bits per chunk, then chunks with starts
  long long* red = reinterpret_cast<long long*>(sh + ((TJ + 1 + NC + 2) & ~1));
  const int32_t* lab = a.pop.labels[1 - a.cur];
  const unsigned mask = warp_lanes(tid, NT);
  for (int i = tid; i <= TJ; i += NT) {
    const int j = tile0 - 1 + i;
    labs[i] = (j >= 0 && j < R_new) ? lab[j] : -1;
  }
  __syncthreads();
  // run starts, one ballot per chunk (lanes of a warp take consecutive slots)
  for (int base = 0; base < TJ; base += NT) {
    const int i = base + tid;
    const bool start = i < TJ && labs[i + 1] != labs[i];
    const unsigned b = __ballot_sync(mask, start);
    if ((i & 31) == 0 && i < TJ) bm[i >> 5] = b;
  }
  __syncthreads();
  if (tid < 32) {  // chunks that hold a run start
    const unsigned nzb = __ballot_sync(0xffffffffu, tid < NC && bm[tid] != 0u);
    if (tid == 0) bm[NC] = nzb;
  }
  __syncthreads();
  const unsigned nz = bm[NC];
  FamilyAcc f;
  for (int base = 0; base < TJ; base += NT) {  // the same iterations in every lane of a warp
    const int i = base + tid, j = tile0 + i, c = i >> 5, l = i & 31;
    int eta = 0;
    if (i < TJ && j < R_new && (bm[c] >> l & 1u)) {
      const unsigned above = l == 31 ? 0u : bm[c] & (~0u << (l + 1));
      const unsigned later = c == 31 ? 0u : nz & (~0u << (c + 1));
      int end;
      if (above) {
        end = tile0 + 32 * c + __ffs(above) - 1;
      } else if (later) {
        const int c2 = __ffs(later) - 1;
        end = tile0 + 32 * c2 + __ffs(bm[c2]) - 1;
      } else {
        end = run_end(lab, labs[i + 1], tile0 + TJ, R_new);
      }
      eta = end - j;
      f.add(eta);
    }
    family_size(a.pop, eta, mask);
  }
  family_flush(f, mask, &a.pop.rec[a.t]);
  // the tiles of both launches that hold slots take part
  const int in_main = min(R_new, a.split);
  const int participants = (in_main + a.tj_main - 1) / a.tj_main +
                           (R_new > a.split ? (R_new - a.split + a.tj_tail - 1) / a.tj_tail : 0);
  family_entropy_last(a.pop, &a.pop.rec[a.t], R_new, participants, tid, NT, red);
}

// One tile of the bit-sliced sweep (+-1 couplings): the slots tile0 .. tile0 + TJ - 1
// of the new population (R_new slots), in the dynamic shared memory sm.
template <int L, int W, int NT, int MB>
__device__ __forceinline__ void sweep_tile(const SweepArgs& a, uint32_t* sm, int tile0, int R_new) {
  using S = BitShape<L, W, NT, MB>;
  constexpr int N = S::N, NP = S::NP, TJ = S::TJ;
  uint32_t* sp = sm;                                               // spins [N][W]
  SiteRec* recs = reinterpret_cast<SiteRec*>(sm + (size_t)N * W);  // [N]
  Deferred* queues = reinterpret_cast<Deferred*>(recs + N);        // [NQ][kQueueCap]
  int* slots = reinterpret_cast<int*>(queues + S::NQ * kQueueCap);  // [33 W]: parents, then level counts
  int* rowtab = slots + S::SLOTS;  // [NP][RPP][8]: word offsets of a row and its four neighbour rows, its first site
  const int tid = threadIdx.x, word = tid % W, part = tid / W;
  Deferred* dq = queues + (S::DEFER ? (tid >> 5) * kQueueCap : 0);
  init_tables<L>(a, recs, tid, NT);
  if constexpr (S::DEFER) fill_row_table<L, W, NP>(rowtab, tid, NT);
  for (int i = tid; i < TJ; i += NT) slots[33 * (i >> 5) + (i & 31)] = tile0 + i < R_new ? a.pop.parents[tile0 + i] : -1;
  __syncthreads();
  gather_bits<L, W, NP>(a, sp, slots, word, part);
  __syncthreads();
  for (int i = tid; i < S::SLOTS; i += NT) slots[i] = 0;
  __syncthreads();

  // sweeps: partition `part` owns rows of parity class p = (y + z) & 1; in
  // half-sweep c its colour sites sit at x = p ^ c mod 2 in every row.
  const uint32_t gbase = (uint32_t)((a.slot_base + tile0) >> 5);  // global index of the tile's first word
  const uint32_t g8 = 8u * (gbase + (uint32_t)word);             // Philox group of block 0 of this word
  const int pclass = part / (NP / 2);
  uint32_t* spw = sp + word;
  for (int s = 0; s < a.n_sweeps; ++s) {
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const uint32_t q = 2u * (uint32_t)s + (uint32_t)c;
      if constexpr (S::DEFER) {
        const ThreadPhilox tp[2] = {thread_philox(g8, q, a.k0, a.k1), thread_philox(g8 + 1u, q, a.k0, a.k1)};
        if ((pclass ^ c) == 0)  // the same in every lane of the warp
          sweep_rows_bits_dq<L, W, NP, 0>(sp, word, recs, part, pclass, tp, q, gbase, dq, rowtab, a);
        else
          sweep_rows_bits_dq<L, W, NP, 1>(sp, word, recs, part, pclass, tp, q, gbase, dq, rowtab, a);
      } else {
        const ThreadPhilox tp[4] = {thread_philox(g8, q, a.k0, a.k1), thread_philox(g8 + 1u, q, a.k0, a.k1),
                                    thread_philox(g8 + 2u, q, a.k0, a.k1), thread_philox(g8 + 3u, q, a.k0, a.k1)};
        if ((pclass ^ c) == 0)
          sweep_rows_bits<L, W, NP, 0>(spw, recs, part, pclass, tp, q, g8, a);
        else
          sweep_rows_bits<L, W, NP, 1>(spw, recs, part, pclass, tp, q, g8, a);
      }
      __syncthreads();
    }
  }
  count_levels_bits<L, W, NP, S::CB>(sp, recs, slots, word, part);
  __syncthreads();
  publish_levels<TJ>(a, slots, tile0, R_new, tid, NT);
  store_bits<L, W, NP>(a, sp, tile0, word, part);
  if (!a.fam) return;
  __syncthreads();  // every shared array is dead now: the family pass takes the space
  tile_families<TJ, NT>(a, reinterpret_cast<int*>(sm), tile0, R_new, tid);
}

// Bit-sliced sweep kernel (+-1 couplings): one tile per CTA.
template <int L, int W, int NT, int MB>
__global__ void __launch_bounds__(NT, MB) k_sweep(const __grid_constant__ SweepArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int R_new = a.pop.rec[a.t].R_tilde;
  const int tile0 = a.tile_base + blockIdx.x * BitShape<L, W, NT, MB>::TJ;
  if (tile0 >= R_new) return;
  sweep_tile<L, W, NT, MB>(a, sm, tile0, R_new);
}

// The sweep arguments of population P at step t from buffer cur with thresholds
// thr (dE = 4, 8, 12), as launch_sweep sets them for a run of one launch.
__host__ __device__ inline void fill_sweep_args(SweepArgs& a, const PopDev& P, const uint32_t* jtab, int64_t pitch,
                                                int n_levels, int t, int cur, int n_sweeps, int tj,
                                                const uint32_t thr[3]) {
  a.pop = P;
  uint32_t k0 = P.key_met[0], k1 = P.key_met[1];
  for (int r = 0; r < 10; ++r) {
    a.k0[r] = k0;
    a.k1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  a.jtab = jtab;
  a.pitch = pitch;
  a.n_levels = n_levels;
  a.t = t;
  a.cur = cur;
  a.n_sweeps = n_sweeps;
  a.slot_base = 0;
  a.fam = 1;
  a.tile_base = 0;
  a.split = 0x7fffffff;
  a.tj_main = tj;
  a.tj_tail = tj;
  a.thr4 = thr[0];
  a.thr8 = thr[1];
  a.thr12 = thr[2];
  const uint32_t thr_u[3] = {thr[2], thr[1], thr[0]};  // u = 0, 1, 2: dE = 12, 8, 4
  for (int p = 0; p < 32; ++p) {
    uint32_t T[3];
    for (int u = 0; u < 3; ++u) T[u] = ((thr_u[u] >> (31 - p)) & 1u) ? ~0u : 0u;
    a.tm[p][0] = T[0];
    a.tm[p][1] = T[0] ^ T[1];
    a.tm[p][2] = T[0] ^ T[2];
    a.tm[p][3] = 0u;
  }
  uint32_t live[3];
  for (int u = 0; u < 3; ++u) live[u] = thr_u[u] ? ~0u : 0u;
  a.live[0] = live[0];
  a.live[1] = live[0] ^ live[1];
  a.live[2] = live[0] ^ live[2];
  a.live[3] = 0u;
}

// The sweeps of a batch's units of one lattice size and launch shape: unit list[k]
// takes the CTAs off[k] .. off[k+1]-1, one tile each; each CTA builds its unit's
// arguments for the round's step in shared memory.
template <int L, int W, int NT, int MB>
__global__ void __launch_bounds__(NT, MB)
    k_sweep_group(const GroupUnit* __restrict__ units, const int32_t* __restrict__ list,
                  const int32_t* __restrict__ off, int n, const int32_t* __restrict__ round) {
  constexpr int TJ = BitShape<L, W, NT, MB>::TJ;
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ SweepArgs sa;
  __shared__ int hdr[3];  // unit, tile0, R_new (tile0 < 0: nothing to do)
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const GroupUnit& u = units[list[lo]];
    const int r = *round, t = u.t0 + 1 + r;
    const int tile0 = (b - off[lo]) * TJ;
    const int R_new = t <= u.last_t ? u.P.rec[t].R_tilde : 0;
    hdr[0] = list[lo];
    hdr[1] = tile0 < R_new ? tile0 : -1;
    hdr[2] = R_new;
    if (tile0 < R_new) {
      const GroupStep& st = u.steps[t];
      fill_sweep_args(sa, u.P, u.jtab, u.g.pitch, u.g.n_levels, t, u.cur0 ^ (r & 1), st.n_sweeps, TJ, st.thr);
    }
  }
  __syncthreads();
  if (hdr[1] < 0) return;
  sweep_tile<L, W, NT, MB>(sa, sm, hdr[1], hdr[2]);
}

template <int L, int W, int NT, int MB>
static int launch_group_t(const GroupUnit* units, const int32_t* list, const int32_t* off, int n, int n_blocks,
                          const int32_t* round, cudaStream_t s) {
  using S = BitShape<L, W, NT, MB>;
  static std::atomic<int> done[64];
  const cudaError_t e = smem_limit_once(k_sweep_group<L, W, NT, MB>, (int)S::SMEM, done);
  if (e != cudaSuccess) return (int)e;
  if (n_blocks <= 0) return 0;
  k_sweep_group<L, W, NT, MB><<<n_blocks, NT, S::SMEM, s>>>(units, list, off, n, round);
  return (int)cudaGetLastError();
}

// ---- Gaussian couplings (§II.A): nibble tiles (eight replicas per word, four
// bits each: gather_tile, store_tile) and one Philox block per site for the eight
// replicas of a word, whose 16-bit halves are the upper halves of their 32-bit
// uniforms (sweep_rows_g).  The acceptance comes from a per-site table built on the
// host for the step's beta: for each of the 64 patterns of antiparallel neighbours
// (bit k: bond k, in the order x+1, x-1, y+1, y-1, z+1, z-1) the threshold of the
// flip, 0xFFFFFFFF when it costs dE <= 0 (always taken) and otherwise
// min(floor(2^32 exp(-beta dE)), 2^32 - 2); the flip is taken when the uniform is
// below it.  Energies are recounted from scratch after the sweeps:
// E = -sum J + 2 sum over antiparallel bonds of J (exact integers).

struct GSweepArgs {
  SweepArgs base;
  const uint32_t* gtab;   // [N][64] acceptance thresholds of this step
  const int32_t* Jq;      // [3N] fixed-point couplings of the forward bonds
  long long Jtot;         // sum of all couplings
};

// The Metropolis uniform U of a replica (Gaussian couplings): its upper 16 bits are
// half (slot & 1) of word (slot >> 1) & 3 of the Philox block at counter
// (h, q, slot >> 3, t) (one block per site for the eight replicas of a nibble word),
// its lower 16 bits the upper half of word slot & 3 at counter (h, q, (slot >> 2) | 2^31,
// t).  With u = the upper half in place, U < thr holds for sure when (u | 0xffff) <
// thr and fails for sure when u >= thr; only in between (probability 2^-16 per
// update) is the second word drawn (g_tie_word).
__device__ __noinline__ uint32_t g_tie_word(uint32_t h, uint32_t q, uint32_t slot, uint32_t t, uint32_t k0,
                                            uint32_t k1) {
  return word_of(philox4x32_10(make_uint4(h, q, (slot >> 2) | 0x80000000u, t), k0, k1), (int)(slot & 3u)) >> 16;
}

template <int L, int W, int NP, int X0>
__device__ __forceinline__ void sweep_rows_g(uint32_t* sp, const SiteRec* recs, int part, const int* rowtab,
                                             const ThreadPhilox& tp, const uint32_t* k0, const uint32_t* k1,
                                             const uint32_t* __restrict__ gtab, uint32_t slot0, uint32_t q,
                                             uint32_t t) {
  constexpr int H = L / 2, RPP = L * L / NP;
#pragma unroll 1
  for (int k = 0; k < RPP; ++k) {
    const int4 e0 = *reinterpret_cast<const int4*>(rowtab + 8 * (part * RPP + k));
    const int rL = rowtab[8 * (part * RPP + k) + 4];  // the row's first site
    uint32_t* p0 = sp + e0.x;
    const uint32_t* pyp = sp + e0.y;
    const uint32_t* pym = sp + e0.z;
    const uint32_t* pzp = sp + e0.w;
    const uint32_t* pzm = sp + rowtab[8 * (part * RPP + k) + 5];
    uint32_t row[L];
#pragma unroll
    for (int x = 0; x < L; ++x) row[x] = p0[x * W];
#pragma unroll
    for (int xh = 0; xh < H; ++xh) {
      const int x = 2 * xh + X0;
      const int xp = x == L - 1 ? 0 : x + 1;
      const int xm = x == 0 ? L - 1 : x - 1;
      const uint32_t h = (uint32_t)rL / 2u + (uint32_t)xh;
      uint32_t w4[4];
      philox_block(kM0 * h, recs[rL + x], tp, k0, k1, w4);
      const uint32_t s0 = row[x];
      const uint32_t P1 = (s0 ^ row[xp]) | ((s0 ^ row[xm]) << 1) | ((s0 ^ pyp[x * W]) << 2);
      const uint32_t P2 = (s0 ^ pym[x * W]) | ((s0 ^ pzp[x * W]) << 1) | ((s0 ^ pzm[x * W]) << 2);
      const uint32_t* tb = gtab + (size_t)(rL + x) * kGPatterns;
      // byte k of Qe (Qo) is the pattern of replica 2k (2k + 1): its P1 bits, then its P2 bits
      const uint32_t Qe = (P1 & 0x0F0F0F0Fu) | ((P2 & 0x0F0F0F0Fu) << 3);
      const uint32_t Qo = ((P1 >> 4) & 0x0F0F0F0Fu) | (((P2 >> 4) & 0x0F0F0F0Fu) << 3);
      uint32_t flip = 0, tie = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint32_t b = __byte_perm((i & 1) ? Qo : Qe, 0u, 0x4440u + (uint32_t)(i >> 1));  // the replica's pattern
        const uint32_t thr = __ldg(tb + b);
        const uint32_t u = (i & 1) ? (w4[i >> 1] & 0xffff0000u) : (w4[i >> 1] << 16);
        // a flip with dE <= 0 (thr = 0xFFFFFFFF) passes here unless u = 0xFFFF0000,
        // which the tie path takes
        if ((u | 0xffffu) < thr) flip |= 1u << (4 * i);
        else if (u < thr) tie |= 1u << i;
      }
      while (tie) {  // rare: the lower 16 bits decide
        const int i = __ffs(tie) - 1;
        tie &= tie - 1;
        const uint32_t b = ((P1 >> (4 * i)) & 7u) | (((P2 >> (4 * i)) & 7u) << 3);
        const uint32_t u = (i & 1) ? (w4[i >> 1] & 0xffff0000u) : (w4[i >> 1] << 16);
        const uint32_t thr = __ldg(tb + b);
        if (thr == 0xFFFFFFFFu || (u | g_tie_word(h, q, slot0 + (uint32_t)i, t, k0[0], k1[0])) < thr)
          flip |= 1u << (4 * i);
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
  int* rowtab = reinterpret_cast<int*>(ecnt + TJ);  // [NP][RPP][8], as the +-1 kernel's
  const int R_new = a.pop.rec[a.t].R_tilde;
  const int tile0 = blockIdx.x * TJ;
  if (tile0 >= R_new) return;
  const int tid = threadIdx.x, word = tid % W, part = tid / W;
  init_tables<L>(a, recs, tid, NT);
  fill_row_table<L, W, NP>(rowtab, tid, NT);
  for (int i = tid; i < TJ; i += NT) ecnt[i] = 0;
  gather_tile<L, W, NP>(a, sp, tile0, R_new, word, part);
  __syncthreads();
  const uint32_t slot0 = (uint32_t)tile0 + 8u * (uint32_t)word;  // the word's first replica
  const uint32_t g = slot0 >> 3;                                     // Philox group of its eight replicas
  const int pclass = part / (NP / 2);
  uint32_t* spw = sp + word;
  for (int s = 0; s < a.n_sweeps; ++s) {
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const uint32_t q = 2u * (uint32_t)s + (uint32_t)c;
      const ThreadPhilox tp = thread_philox(g, q, a.k0, a.k1);
      if ((pclass ^ c) == 0)
        sweep_rows_g<L, W, NP, 0>(spw, recs, part, rowtab, tp, a.k0, a.k1, ga.gtab, slot0, q, (uint32_t)a.t);
      else
        sweep_rows_g<L, W, NP, 1>(spw, recs, part, rowtab, tp, a.k0, a.k1, ga.gtab, slot0, q, (uint32_t)a.t);
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
  const size_t smem = S::SMEM + (size_t)S::TJ * 4 + S::SMEM_ROWS;  // energy counters are 8 bytes, not 4
  static std::atomic<int> done[64];
  const cudaError_t e = smem_limit_once(k_sweep_g<L, W, NT, MB>, (int)smem, done);
  if (e != cudaSuccess) return (int)e;
  dim3 grid((unsigned)((g.R_cap + S::TJ - 1) / S::TJ));
  k_sweep_g<L, W, NT, MB><<<grid, NT, smem, s>>>(args);
  return (int)cudaGetLastError();
}

template <int L, int W, int NT, int MB>
static int launch_t(const RunGeom& g, const SweepArgs& args, cudaStream_t s) {
  using S = BitShape<L, W, NT, MB>;
  static std::atomic<int> done[64];
  const cudaError_t e = smem_limit_once(k_sweep<L, W, NT, MB>, (int)S::SMEM, done);
  if (e != cudaSuccess) return (int)e;
  // tiles from tile_base up to the split (main launch) or to the capacity (tail launch)
  const int64_t end = args.tile_base < args.split ? std::min<int64_t>(args.split, g.R_cap) : g.R_cap;
  if (end <= args.tile_base) return 0;
  dim3 grid((unsigned)((end - args.tile_base + S::TJ - 1) / S::TJ));
  k_sweep<L, W, NT, MB><<<grid, NT, S::SMEM, s>>>(args);
  return (int)cudaGetLastError();
}

namespace {

// Candidate launch shapes of the +-1 sweep: words per site row W (32W replicas
// per tile), threads per CTA, CTAs per SM the kernel is compiled for (its
// register cap).  The first entry of each L is the default; the autotuner may
// pick another, and a run too small to give every SM a tile takes the shape
// with the most tiles (the W = 8 entries exist for those).  All give identical
// results.  At L = 14 the partitions of a
// warp may straddle the two parity classes (it then runs both colour offsets).
struct ShapeEntry {
  int L, W, NT, MB;
  size_t smem;
  int (*launch)(const RunGeom&, const SweepArgs&, cudaStream_t);
  int (*launch_group)(const GroupUnit*, const int32_t*, const int32_t*, int, int, const int32_t*, cudaStream_t);
};
#define PA_SHAPE(L, W, NT, MB) \
  {L, W, NT, MB, BitShape<L, W, NT, MB>::SMEM, &launch_t<L, W, NT, MB>, &launch_group_t<L, W, NT, MB>}
const ShapeEntry kShapes[] = {
    PA_SHAPE(2, 32, 128, 1),   PA_SHAPE(2, 32, 64, 2),
    PA_SHAPE(4, 32, 256, 2),   PA_SHAPE(4, 32, 128, 4),  PA_SHAPE(4, 32, 512, 1),  PA_SHAPE(4, 8, 128, 4),
    PA_SHAPE(6, 32, 384, 2),   PA_SHAPE(6, 32, 192, 4),  PA_SHAPE(6, 32, 576, 1),  PA_SHAPE(6, 8, 288, 2),
    PA_SHAPE(8, 32, 256, 2),   PA_SHAPE(8, 32, 512, 1),  PA_SHAPE(8, 16, 256, 2),  PA_SHAPE(8, 8, 256, 2),
    PA_SHAPE(10, 32, 640, 1),  PA_SHAPE(10, 16, 320, 2), PA_SHAPE(10, 8, 160, 3),
    PA_SHAPE(12, 16, 576, 1),  PA_SHAPE(12, 16, 768, 1), PA_SHAPE(12, 8, 384, 2),
    PA_SHAPE(14, 8, 784, 1),   PA_SHAPE(14, 8, 224, 1),  PA_SHAPE(14, 4, 392, 1),
    PA_SHAPE(16, 4, 512, 1),   PA_SHAPE(16, 4, 256, 1),
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
  const ShapeEntry* tail = g.tail_shape >= 0 ? shape_of(g.L, g.tail_shape) : nullptr;
  for (int i = 0; i < g.n_pop; ++i) {
    SweepArgs args;
    fill_sweep_args(args, pops[i], jtab, g.pitch, g.n_levels, t, cur, n_sweeps, 32 * shape->W, met_thr);
    args.slot_base = g.slot_base;
    args.fam = g.shard ? 0 : 1;
    args.split = tail ? g.tail_from : 0x7fffffff;
    args.tj_tail = tail ? 32 * tail->W : 32 * shape->W;
    int e = shape->launch(g, args, s);
    if (e == 0 && tail) {
      args.tile_base = g.tail_from;
      e = tail->launch(g, args, s);
    }
    if (e != 0) return e;
  }
  return 0;
}

int sweep_tile_slots(int L, int shape) {
  const ShapeEntry* e = shape_of(L, shape);
  return e ? 32 * e->W : 0;
}

int launch_group_sweep(int L, int shape, const GroupUnit* units, const int32_t* list, const int32_t* off, int n,
                       int n_blocks, const int32_t* round, void* stream) {
  const ShapeEntry* e = shape_of(L, shape);
  if (!e || n <= 0) return (int)cudaErrorInvalidValue;
  return e->launch_group(units, list, off, n, n_blocks, round, (cudaStream_t)stream);
}

void sweep_tail_plan(int L, int shape, int64_t R, int n_sm, int32_t* tail_shape, int32_t* tail_from) {
  *tail_shape = -1;
  *tail_from = 0;
  const ShapeEntry* m = shape_of(L, shape);
  if (!m || n_sm <= 0) return;
  const int64_t tj = 32LL * m->W, slots = (int64_t)n_sm * m->MB, tiles = (R + tj - 1) / tj;
  const int64_t full = tiles / slots, rest = tiles - full * slots;
  if (full < 1 || rest == 0 || 10 * rest > 6 * slots) return;  // the last wave is more than 60 % full
  int best = -1;
  for (int i = 0; i < sweep_shape_count(L); ++i) {  // the largest smaller tile
    const ShapeEntry* e = shape_of(L, i);
    if (e->W < m->W && (best < 0 || e->W > shape_of(L, best)->W)) best = i;
  }
  if (best < 0) return;
  *tail_shape = best;
  *tail_from = (int32_t)(full * slots * tj);
}

int launch_g_sweep(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, const int32_t* Jq, long long Jtot,
                   const uint32_t* gtab, int t, int n_sweeps, void* stream) {
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
    args.slot_base = 0;
    args.fam = 0;
    args.tile_base = 0;
    args.split = 0x7fffffff;
    args.tj_main = args.tj_tail = 1;
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
