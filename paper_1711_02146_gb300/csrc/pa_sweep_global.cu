// pa_sweep_global.cu — the sweep for lattices too large for a tile in shared
// memory (16 < L <= 64, +-1 couplings).  The resampled population is first
// copied from its parents (replica copy, §II), then every half-sweep is one
// launch that updates all sites of one colour of every replica in place in
// global memory; the energy levels are counted afterwards by k_levels_and_hist.
//
// Layout as everywhere: int8 spins +1 = 0x01 / -1 = 0xFF, site-major rows of
// pitch bytes, so one 32-bit word holds four replicas of one site and one thread
// updates those four with one Philox4x32-10 block: counter (n >> 1, 2s + c,
// j >> 2, t), word j & 3 for slot j (the stream every other sweep uses).
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

// One half-sweep (colour c of sweep s) of every replica, four replicas per thread.
__global__ void __launch_bounds__(kThreads) k_sweep_global(RunGeom g, PopDev P, int buf, const uint32_t* __restrict__ jtab,
                                                           int t, int s, int c, uint32_t thr4, uint32_t thr8,
                                                           uint32_t thr12, int64_t words) {
  const int R = P.rec[t].R_tilde;
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int H = g.L / 2;
  if (idx >= words * (int64_t)(g.N / 2)) return;
  const int gs = (int)(idx / words);  // colour site: row r, half-index xh
  const int wi = (int)(idx % words);
  if (4 * wi >= R) return;
  const int L = g.L;
  const int r = gs / H, xh = gs % H;
  const int y = r % L, z = r / L;
  const int x = 2 * xh + ((c + y + z) & 1);
  const int n = x + L * r;
  const int xp = (x + 1 == L ? 0 : x + 1) + L * r, xm = (x == 0 ? L - 1 : x - 1) + L * r;
  const int yp = x + L * ((y + 1 == L ? 0 : y + 1) + L * z), ym = x + L * ((y == 0 ? L - 1 : y - 1) + L * z);
  const int zp = x + L * (y + L * (z + 1 == L ? 0 : z + 1)), zm = x + L * (y + L * (z == 0 ? L - 1 : z - 1));
  const int64_t pw = g.pitch / 4;
  uint32_t* S = reinterpret_cast<uint32_t*>(P.spins[buf]);
  const uint32_t s0 = S[n * pw + wi];
  // twice the unsatisfied bonds of each replica, one byte each
  const uint32_t u2 = ((s0 ^ S[xp * pw + wi] ^ jtab[4 * n + 0]) & kBit1) +
                      ((s0 ^ S[xm * pw + wi] ^ jtab[4 * xm + 0]) & kBit1) +
                      ((s0 ^ S[yp * pw + wi] ^ jtab[4 * n + 1]) & kBit1) +
                      ((s0 ^ S[ym * pw + wi] ^ jtab[4 * ym + 1]) & kBit1) +
                      ((s0 ^ S[zp * pw + wi] ^ jtab[4 * n + 2]) & kBit1) +
                      ((s0 ^ S[zm * pw + wi] ^ jtab[4 * zm + 2]) & kBit1);
  const uint4 rw = philox4x32_10(make_uint4((uint32_t)(n >> 1), (uint32_t)(2 * s + c), (uint32_t)wi, (uint32_t)t),
                                 P.key_met[0], P.key_met[1]);
  uint32_t flip = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint32_t u = (u2 >> (8 * b + 1)) & 0xFu;  // 0..6; flipping costs dE = 12 - 4u
    const uint32_t thr = u == 2 ? thr4 : u == 1 ? thr8 : u == 0 ? thr12 : 0u;
    if (u >= 3 || word_of(rw, b) < thr) flip |= 0xFEu << (8 * b);
  }
  S[n * pw + wi] = s0 ^ flip;
}

}  // namespace

bool lattice_supported(int L) { return L >= 2 && L <= kMaxLGlobal && L % 2 == 0; }

int launch_sweep_global(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, int t, int n_sweeps,
                        const uint32_t met_thr[3], void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t words = (g.R_cap + 3) / 4;
  for (int p = 0; p < g.n_pop; ++p) {
    const int64_t copy_threads = words * g.N;
    k_copy_parents<<<(unsigned)((copy_threads + kThreads - 1) / kThreads), kThreads, 0, st>>>(g, pops[p], cur, t,
                                                                                              words);
    const int64_t half = words * (int64_t)(g.N / 2);
    for (int s = 0; s < n_sweeps; ++s)
      for (int c = 0; c < 2; ++c)
        k_sweep_global<<<(unsigned)((half + kThreads - 1) / kThreads), kThreads, 0, st>>>(
            g, pops[p], 1 - cur, jtab, t, s, c, met_thr[0], met_thr[1], met_thr[2], words);
    const int e = (int)cudaGetLastError();
    if (e) return e;
  }
  return launch_levels_and_hist(g, pops, 1 - cur, jtab, t, stream);
}

}  // namespace pa
