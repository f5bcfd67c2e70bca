// pa_sweep.cu — the Metropolis sweep kernel (the dominant cost of a PA step).
//
// One CTA owns a tile of TJ = 4W consecutive slots of the NEW population and
// all N sites of those replicas in shared memory (W 32-bit words per site row,
// four int8 replicas per word).  It
//   1. gathers each slot's spins from its parent in the old population (the
//      replica copy of the resampling, §II, fused into the load),
//   2. runs S checkerboard Metropolis sweeps at beta_t in shared memory (colour
//      c = (x + y + z) & 1, colour 0 then colour 1; neighbours of a site all
//      have the other colour, so every site of a colour updates independently),
//   3. counts each replica's unsatisfied bonds (its energy level k), adds the
//      tile to the level histogram of step t, and
//   4. writes the tile to the new population buffer.
// HBM traffic is one read and one write of the tile per step, whatever S is.
//
// Metropolis rule: flipping s_n costs dE = 2 s_n h_n = 12 - 4u, u = unsatisfied
// bonds at n.  It is accepted when u >= 3 (dE <= 0) or when the Philox word r
// is below thr[dE/4 - 1] = floor(2^32 exp(-beta dE)).  r is word (j & 3) of
// Philox4x32-10 at counter (n >> 1, 2s + c, j >> 2, t) keyed by (run_seed,
// Metropolis, population): one call serves the four replicas of a word.
#include <cuda_runtime.h>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

struct SweepArgs {
  PopDev pops[2];
  const uint32_t* jtab;  // [N][4] forward-bond XOR masks
  int64_t pitch;
  int32_t n_levels;
  int32_t t;
  int32_t cur;
  int32_t n_sweeps;
  uint32_t thr4, thr8, thr12;
};

constexpr uint32_t kBit1Mask = 0x02020202u;

template <int L, int W, int NT>
struct SweepShape {
  static constexpr int N = L * L * L;
  static constexpr int ROWS = L * L;
  static constexpr int NP = NT / W;  // row partitions
  static constexpr int TJ = 4 * W;   // replicas per tile
  static constexpr size_t SMEM = (size_t)N * W * 4 + (size_t)N * 16 + (size_t)TJ * 4;
  static_assert(NT % W == 0, "threads must tile the words of a row");
};

template <int L, int W, int NT>
__global__ void __launch_bounds__(NT) k_sweep(SweepArgs a) {
  using S = SweepShape<L, W, NT>;
  constexpr int N = S::N, NP = S::NP, TJ = S::TJ, ROWS = S::ROWS;
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* sp = sm;                       // spins [N][W]
  uint32_t* jt = sm + N * W;               // coupling masks [N][4]
  int* ecnt = reinterpret_cast<int*>(jt + 4 * N);  // [TJ] unsatisfied-bond counts (x2)

  const int pop = blockIdx.y;
  const PopDev& P = a.pops[pop];
  const int R_new = P.rec[a.t].R_tilde;
  const int tile0 = blockIdx.x * TJ;
  if (tile0 >= R_new) return;
  const int tid = threadIdx.x;
  const int word = tid % W;
  const int part = tid / W;

  for (int i = tid; i < 4 * N; i += NT) jt[i] = a.jtab[i];
  for (int i = tid; i < TJ; i += NT) ecnt[i] = 0;

  // 1. gather from the parents
  int par[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = tile0 + 4 * word + b;
    par[b] = j < R_new ? P.parents[j] : -1;
  }
  const int8_t* src = P.spins[a.cur];
  for (int n = part; n < N; n += NP) {
    const int8_t* row = src + (size_t)n * a.pitch;
    uint32_t w = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const uint32_t v = par[b] >= 0 ? (uint32_t)(uint8_t)row[par[b]] : 0x01u;
      w |= v << (8 * b);
    }
    sp[n * W + word] = w;
  }
  __syncthreads();

  // 2. sweeps
  const uint32_t k0 = P.key_met[0], k1 = P.key_met[1];
  const uint32_t wordidx = (uint32_t)(tile0 >> 2) + (uint32_t)word;
  const uint32_t T4 = a.thr4, T8 = a.thr8, T12 = a.thr12;
  for (int s = 0; s < a.n_sweeps; ++s) {
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const uint32_t ctr1 = 2u * (uint32_t)s + (uint32_t)c;
      for (int r = part; r < ROWS; r += NP) {
        const int y = r % L, z = r / L;
        const int yp = y == L - 1 ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
        const int zp = z == L - 1 ? 0 : z + 1, zm = z == 0 ? L - 1 : z - 1;
        const int b0 = r * L;
        const int byp = (yp + L * z) * L, bym = (ym + L * z) * L;
        const int bzp = (y + L * zp) * L, bzm = (y + L * zm) * L;
        const int x0 = (y + z + c) & 1;
#pragma unroll
        for (int xh = 0; xh < L / 2; ++xh) {
          const int x = 2 * xh + x0;
          const int xp = x == L - 1 ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
          const int n = b0 + x;
          const uint32_t s0 = sp[n * W + word];
          const uint32_t u2 = ((s0 ^ sp[(b0 + xp) * W + word] ^ jt[4 * n + 0]) & kBit1Mask) +
                              ((s0 ^ sp[(b0 + xm) * W + word] ^ jt[4 * (b0 + xm) + 0]) & kBit1Mask) +
                              ((s0 ^ sp[(byp + x) * W + word] ^ jt[4 * n + 1]) & kBit1Mask) +
                              ((s0 ^ sp[(bym + x) * W + word] ^ jt[4 * (bym + x) + 1]) & kBit1Mask) +
                              ((s0 ^ sp[(bzp + x) * W + word] ^ jt[4 * n + 2]) & kBit1Mask) +
                              ((s0 ^ sp[(bzm + x) * W + word] ^ jt[4 * (bzm + x) + 2]) & kBit1Mask);
          const uint4 rr = philox4x32_10(make_uint4((uint32_t)n >> 1, ctr1, wordidx, (uint32_t)a.t), k0, k1);
          uint32_t fm = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const uint32_t u = (u2 >> (8 * b + 1)) & 7u;
            const uint32_t rb = word_of(rr, b);
            const bool acc = (u >= 3u) || (u == 2u ? rb < T4 : (u == 1u ? rb < T8 : rb < T12));
            fm |= acc ? (0xFEu << (8 * b)) : 0u;
          }
          sp[n * W + word] = s0 ^ fm;
        }
      }
      __syncthreads();
    }
  }

  // 3. energy levels: unsatisfied forward bonds of every site of the replicas
  {
    int cnt[4] = {0, 0, 0, 0};
    for (int r = part; r < ROWS; r += NP) {
      const int y = r % L, z = r / L;
      const int yp = y == L - 1 ? 0 : y + 1, zp = z == L - 1 ? 0 : z + 1;
      const int b0 = r * L, byp = (yp + L * z) * L, bzp = (y + L * zp) * L;
      uint32_t acc = 0;  // <= 6L per byte
#pragma unroll
      for (int x = 0; x < L; ++x) {
        const int xp = x == L - 1 ? 0 : x + 1;
        const int n = b0 + x;
        const uint32_t s0 = sp[n * W + word];
        acc += ((s0 ^ sp[(b0 + xp) * W + word] ^ jt[4 * n + 0]) & kBit1Mask) +
               ((s0 ^ sp[(byp + x) * W + word] ^ jt[4 * n + 1]) & kBit1Mask) +
               ((s0 ^ sp[(bzp + x) * W + word] ^ jt[4 * n + 2]) & kBit1Mask);
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
      const int k = ecnt[i] >> 1;
      P.levels[j] = k;
      atomicAdd(&hist[k], 1u);
    }
  }

  // 4. store the tile
  uint32_t* dst = reinterpret_cast<uint32_t*>(P.spins[1 - a.cur]);
  const int64_t pw = a.pitch / 4;
  for (int n = part; n < N; n += NP) dst[n * pw + (tile0 >> 2) + word] = sp[n * W + word];
}

template <int L, int W, int NT>
static int launch_t(const RunGeom& g, const SweepArgs& args, cudaStream_t s) {
  using S = SweepShape<L, W, NT>;
  cudaError_t e = cudaFuncSetAttribute(k_sweep<L, W, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
  if (e != cudaSuccess) return (int)e;
  dim3 grid((unsigned)((g.R_cap + S::TJ - 1) / S::TJ), (unsigned)g.n_pop);
  k_sweep<L, W, NT><<<grid, NT, S::SMEM, s>>>(args);
  return (int)cudaGetLastError();
}

bool sweep_supported(int L) { return L >= 2 && L <= kMaxL && L % 2 == 0; }

int launch_sweep(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, int t, int n_sweeps,
                 const uint32_t met_thr[3], void* stream) {
  SweepArgs args;
  for (int i = 0; i < g.n_pop && i < 2; ++i) args.pops[i] = pops[i];
  args.jtab = jtab;
  args.pitch = g.pitch;
  args.n_levels = g.n_levels;
  args.t = t;
  args.cur = cur;
  args.n_sweeps = n_sweeps;
  args.thr4 = met_thr[0];
  args.thr8 = met_thr[1];
  args.thr12 = met_thr[2];
  cudaStream_t s = (cudaStream_t)stream;
  switch (g.L) {
    case 2: return launch_t<2, 32, 128>(g, args, s);
    case 4: return launch_t<4, 32, 256>(g, args, s);
    case 6: return launch_t<6, 32, 384>(g, args, s);
    case 8: return launch_t<8, 32, 512>(g, args, s);
    case 10: return launch_t<10, 32, 640>(g, args, s);
    case 12: return launch_t<12, 16, 576>(g, args, s);
    case 14: return launch_t<14, 8, 224>(g, args, s);
    case 16: return launch_t<16, 8, 256>(g, args, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace pa
