// pa_sweep_global.cu — the sweep for lattices too large for a tile in shared
// memory (16 < L <= 64, +-1 couplings).  The resampled population is first
// copied from its parents (replica copy, §II), then every half-sweep is one
// launch that updates all sites of one colour of every replica in place in
// global memory; the energy levels are counted afterwards by k_levels_and_hist.
//
// Layout as everywhere: int8 spins +1 = 0x01 / -1 = 0xFF, site-major rows of
// pitch bytes; one thread updates eight replicas (one 64-bit word) of one site.
// The acceptance test is the tile kernel's: a replica's 32-bit uniform is its bit
// column (bit 31 - p is bit j & 31 of word p & 3 of Philox4x32-10 at counter
// (n >> 1, 2s + c, 8 (j >> 5) + p / 4, t)), compared with its threshold from the
// top bit down until the first differing bit; the thread draws blocks until its
// eight replicas are decided.
#include <cuda_runtime.h>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

constexpr uint32_t kBit1 = 0x02020202u;  // bit 1 of each byte: 1 for an unsatisfied bond term
constexpr int kThreads = 256;

// new[n][j] = old[n][parents[j]] for every site n and new slot j < R~_t.
__global__ void __launch_bounds__(kThreads) k_copy_parents(RunGeom g, PopDev P, int cur, int t, int64_t words) {
  const int R = P.rec[t].R_tilde;
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (idx >= words * g.N) return;
  const int n = (int)(idx / words);
  const int wi = (int)(idx % words);
  const int j0 = 4 * wi;
  if (j0 >= R) return;
  const int8_t* src = P.spins[cur] + (size_t)n * g.pitch;
  int8_t* dst = P.spins[1 - cur] + (size_t)n * g.pitch;
  int p[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) p[b] = j0 + b < R ? P.parents[j0 + b] : -1;
  uint32_t out;
  if (p[0] >= 0 && (p[0] & 3) == 0 && p[1] == p[0] + 1 && p[2] == p[0] + 2 && p[3] == p[0] + 3) {
    out = *reinterpret_cast<const uint32_t*>(src + p[0]);  // four consecutive parents
  } else {
    out = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) out |= (uint32_t)(uint8_t)(p[b] >= 0 ? src[p[b]] : (int8_t)1) << (8 * b);
  }
  *reinterpret_cast<uint32_t*>(dst + (size_t)j0) = out;
}

// Twice the unsatisfied bonds of each of four replicas (one byte each) of site n.
__device__ __forceinline__ uint32_t unsatisfied2(uint32_t s0, uint32_t sxp, uint32_t sxm, uint32_t syp, uint32_t sym,
                                                 uint32_t szp, uint32_t szm, uint32_t jxp, uint32_t jxm, uint32_t jyp,
                                                 uint32_t jym, uint32_t jzp, uint32_t jzm) {
  return ((s0 ^ sxp ^ jxp) & kBit1) + ((s0 ^ sxm ^ jxm) & kBit1) + ((s0 ^ syp ^ jyp) & kBit1) +
         ((s0 ^ sym ^ jym) & kBit1) + ((s0 ^ szp ^ jzp) & kBit1) + ((s0 ^ szm ^ jzm) & kBit1);
}

// One half-sweep (colour c of sweep s) of every replica, eight replicas per thread.
__global__ void __launch_bounds__(kThreads) k_sweep_global(RunGeom g, PopDev P, int buf, const uint32_t* __restrict__ jtab,
                                                           int t, int s, int c, uint32_t thr4, uint32_t thr8,
                                                           uint32_t thr12, int64_t words) {
  const int R = P.rec[t].R_tilde;
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int H = g.L / 2;
  if (idx >= words * (int64_t)(g.N / 2)) return;
  const int gs = (int)(idx / words);  // colour site: row r, half-index xh
  const int wi = (int)(idx % words);
  if (8 * wi >= R) return;
  const int L = g.L;
  const int r = gs / H, xh = gs % H;
  const int y = r % L, z = r / L;
  const int x = 2 * xh + ((c + y + z) & 1);
  const int n = x + L * r;
  const int xp = (x + 1 == L ? 0 : x + 1) + L * r, xm = (x == 0 ? L - 1 : x - 1) + L * r;
  const int yp = x + L * ((y + 1 == L ? 0 : y + 1) + L * z), ym = x + L * ((y == 0 ? L - 1 : y - 1) + L * z);
  const int zp = x + L * (y + L * (z + 1 == L ? 0 : z + 1)), zm = x + L * (y + L * (z == 0 ? L - 1 : z - 1));
  const int64_t pw = g.pitch / 8;
  uint2* S = reinterpret_cast<uint2*>(P.spins[buf]);
  const uint2 s0 = S[n * pw + wi], sxp = S[xp * pw + wi], sxm = S[xm * pw + wi], syp = S[yp * pw + wi],
              sym = S[ym * pw + wi], szp = S[zp * pw + wi], szm = S[zm * pw + wi];
  const uint32_t jxp = jtab[4 * n + 0], jxm = jtab[4 * xm + 0], jyp = jtab[4 * n + 1], jym = jtab[4 * ym + 1],
                 jzp = jtab[4 * n + 2], jzm = jtab[4 * zm + 2];
  const uint32_t u2[2] = {unsatisfied2(s0.x, sxp.x, sxm.x, syp.x, sym.x, szp.x, szm.x, jxp, jxm, jyp, jym, jzp, jzm),
                          unsatisfied2(s0.y, sxp.y, sxm.y, syp.y, sym.y, szp.y, szm.y, jxp, jxm, jyp, jym, jzp, jzm)};
  const uint32_t j0 = 8u * (uint32_t)wi, sh = j0 & 31u;  // slots j0 .. j0 + 7: bits sh .. sh + 7 of the words
  uint32_t thr[8], undecided = 0, accept = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t u = (u2[i >> 2] >> (8 * (i & 3) + 1)) & 0xFu;  // 0..6; flipping costs dE = 12 - 4u
    thr[i] = u == 2 ? thr4 : u == 1 ? thr8 : thr12;
    if (u >= 3)
      accept |= 1u << i;
    else if (thr[i] != 0)
      undecided |= 1u << i;
  }
  for (int b = 0; b < 8 && undecided; ++b) {
    const uint4 rw = philox4x32_10(make_uint4((uint32_t)(n >> 1), (uint32_t)(2 * s + c), 8u * (j0 >> 5) + (uint32_t)b,
                                              (uint32_t)t),
                                   P.key_met[0], P.key_met[1]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int p = 4 * b + k;
      const uint32_t bits = word_of(rw, k) >> sh;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint32_t rb = (bits >> i) & 1u, tb = (thr[i] >> (31 - p)) & 1u;
        if (((undecided >> i) & 1u) && rb != tb) {
          undecided &= ~(1u << i);
          if (tb) accept |= 1u << i;
        }
      }
    }
  }
  uint32_t flip[2] = {0u, 0u};
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if ((accept >> i) & 1u) flip[i >> 2] |= 0xFEu << (8 * (i & 3));
  S[n * pw + wi] = make_uint2(s0.x ^ flip[0], s0.y ^ flip[1]);
}

}  // namespace

bool lattice_supported(int L) { return L >= 2 && L <= kMaxLGlobal && L % 2 == 0; }

int launch_copy_parents(const RunGeom& g, PopDev* pops, int pop, int cur, int t, void* stream) {
  const int64_t words = (g.R_cap + 3) / 4;
  k_copy_parents<<<(unsigned)((words * g.N + kThreads - 1) / kThreads), kThreads, 0, (cudaStream_t)stream>>>(
      g, pops[pop], cur, t, words);
  return (int)cudaGetLastError();
}

int launch_sweep_global(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, int t, int n_sweeps,
                        const uint32_t met_thr[3], void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t words = (g.R_cap + 3) / 4, words8 = (g.R_cap + 7) / 8;
  for (int p = 0; p < g.n_pop; ++p) {
    const int64_t copy_threads = words * g.N;
    k_copy_parents<<<(unsigned)((copy_threads + kThreads - 1) / kThreads), kThreads, 0, st>>>(g, pops[p], cur, t,
                                                                                              words);
    const int64_t half = words8 * (int64_t)(g.N / 2);
    for (int s = 0; s < n_sweeps; ++s)
      for (int c = 0; c < 2; ++c)
        k_sweep_global<<<(unsigned)((half + kThreads - 1) / kThreads), kThreads, 0, st>>>(
            g, pops[p], 1 - cur, jtab, t, s, c, met_thr[0], met_thr[1], met_thr[2], words8);
    const int e = (int)cudaGetLastError();
    if (e) return e;
  }
  return launch_levels_and_hist(g, pops, 1 - cur, jtab, t, stream);
}

}  // namespace pa
