// pa_runtime.cpp — host side of the C ABI in include/pa.h.
//
// Owns the device memory of a run, launches the step kernels on the run's
// stream, and finalises observables from the integer records the kernels write.
// The FP64 host parts of the step are here: the Boltzmann weight table of a
// temperature move, the Metropolis thresholds, the adaptive schedule (§IV.B)
// and the estimators of §II.A / §III.A.  Compile with -ffp-contract=off so that
// every expression rounds as written.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

#include "../../include/pa.h"
#include "pa_internal.h"

using pa::PopDev;
using pa::RunGeom;
using pa::StepRec;

struct pa_ctx {
  pa_config cfg{};
  std::vector<double> betas;   // filled as the run advances (adaptive) or at creation
  std::vector<int32_t> sweeps;
  bool adaptive = false;
  RunGeom g{};
  cudaStream_t stream = nullptr;
  int t = 0;
  bool done = false;
  int cur = 0;
  int error = PA_OK;
  int8_t* J = nullptr;          // device [3N]
  uint32_t* jtab = nullptr;     // device [N][4]
  int32_t* status = nullptr;    // device flags
  unsigned long long* qhist = nullptr;  // device [n_temps][q_bins]
  PopDev pops[2]{};
  // Boltzmann weight tables exp(-dbeta 2j), one per distinct dbeta (device)
  std::map<uint64_t, double*> wtables;
  std::vector<double> wtables_host;  // host copy of the explicit schedule's tables (source of their upload)
  double* wadapt = nullptr;     // adaptive schedule: the table of the current step
  double* wadapt_host = nullptr;  // its pinned host copy (uploaded without a wait)
  uint32_t* gtab_host = nullptr;  // pinned host copy of the adaptive Gaussian step's site tables
  int32_t occ_span = -1;          // adaptive +-1: highest minus lowest occupied level of population 0
  // All device buffers of the run are carved from one stream-ordered allocation:
  // a run costs the memory pool one block, so the pool's free list stays short
  // when many runs come and go (a request server).
  char* slab = nullptr;
  size_t slab_bytes = 0;        // sizing pass: running total; carving pass: the slab's size
  size_t slab_used = 0;
  // instrumentation (pa_stats)
  pa_stats stats{};
  bool timing = false;
  std::vector<cudaEvent_t> events;                 // pool
  size_t events_used = 0;
  struct Timed { int phase; cudaEvent_t start, end; };
  std::vector<Timed> timed;
  std::vector<std::pair<int, int>> counted_steps;  // (t, S_t) since the last reset
  // Gaussian-coupling model
  int model = PA_MODEL_PM1;
  int32_t* Jq = nullptr;                 // device [3N] fixed-point couplings
  long long Jtot = 0;                    // sum of the couplings
  uint32_t* gtab = nullptr;              // device [n_temps][N][64] acceptance thresholds
  double* gw = nullptr;                  // device [n_temps][16384] weight tables
  unsigned long long* qlhist = nullptr;  // device [n_temps][q_bins] link-overlap histograms
  double* gbis = nullptr;                // device {lo, hi, mid, state}: the adaptive bisection (Gaussian)
  double* gbt = nullptr;                 // device: its three table sets and chunk sums (one-launch bisection)
  unsigned long long* gbar = nullptr;    // device: that launch's grid barrier words
  int gbis_blocks = -1;                  // blocks of the one-launch bisection (0: launch per halving)
  int gbis_withheld = -1;                // pa_debug_bisect: block kept from the first barrier
  std::vector<int32_t> Jq_host;
  pa::LookbackTest lookback;             // pa_debug_lookback (tests of the bounded wait)
  // Completion events of the last steps (a ring, step u in entry u & 3, -1: none), so
  // that reading step t's results waits for step t only, not for steps issued after
  // it; those reads go through their own stream.
  cudaEvent_t step_ev[4] = {};
  int32_t step_ev_t[4] = {-1, -1, -1, -1};
  cudaStream_t rd = nullptr;
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? PA_OK : PA_ERR_CUDA; }

// The step's sum over families of nu ln nu from its exact 128-bit fixed-point form
// (units of 2^-100), rounded to double once.
double nu_ln_nu(const StepRec& r) {
  const unsigned __int128 u = ((unsigned __int128)(uint64_t)r.nll_hi << 64) | (unsigned __int128)r.nll_lo;
  return (double)(__int128)u * 0x1p-100;
}

// Sweep launch shape selected per device and lattice size (an index among the
// shapes compiled for L; static storage starts at 0, the default shape).
constexpr int kMaxDevices = 64;
std::atomic<int32_t> g_sweep_choice[kMaxDevices][pa::kMaxL + 1];
std::atomic<bool> g_sweep_pinned[kMaxDevices][pa::kMaxL + 1];  // set by pa_sweep_select with an index

// The shape a +-1 run of population capacity R_cap takes: the chosen one, unless it
// was not pinned and the population gives fewer tiles than the device has SMs; then
// the shape of that L with the most tiles (every shape gives identical results).
int run_shape(int L, int64_t R_cap, int dev) {
  const int chosen = g_sweep_choice[dev][L].load();
  if (g_sweep_pinned[dev][L].load()) return chosen;
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return chosen;
  auto tiles = [&](int i) {
    pa::SweepShapeInfo si;
    if (!pa::sweep_shape_info(L, i, &si)) return (int64_t)0;
    const int64_t tj = 32LL * si.W;
    return (R_cap + tj - 1) / tj;
  };
  int best = chosen;
  int64_t best_tiles = tiles(chosen);
  if (best_tiles >= n_sm) return chosen;
  for (int i = 0; i < pa::sweep_shape_count(L); ++i)
    if (tiles(i) > best_tiles) {
      best = i;
      best_tiles = tiles(i);
    }
  return best;
}

int current_device(int* dev) {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return PA_ERR_CUDA;
  *dev = d;
  return PA_OK;
}

// Device memory pool of the runs, one per device, created on first use.  Runs
// allocate from it stream-ordered (one slab each) like from the default pool, but
// with every cross-stream reuse policy off: with hundreds of run streams, checking
// earlier runs' frees for reuse made each allocation take about a millisecond.
// Memory freed on one stream is still reused by later allocations on that stream,
// and by any stream once the free has been seen complete through a synchronisation.
int runs_pool(int dev, cudaMemPool_t* out) {
  static std::mutex mu;
  static cudaMemPool_t pools[kMaxDevices] = {};
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return PA_ERR_CUDA;
    int off = 0;
    for (cudaMemPoolAttr a : {cudaMemPoolReuseFollowEventDependencies, cudaMemPoolReuseAllowOpportunistic,
                              cudaMemPoolReuseAllowInternalDependencies})
      if (cudaMemPoolSetAttribute(p, a, &off) != cudaSuccess) {
        cudaMemPoolDestroy(p);
        return PA_ERR_CUDA;
      }
    pools[dev] = p;
  }
  *out = pools[dev];
  return PA_OK;
}

// Copies are ordered on the run's stream and waited for on that stream only, so
// runs on other streams keep going.
int copy_d2h(pa_ctx* c, void* dst, const void* src, size_t bytes) {
  c->stats.d2h_bytes += (int64_t)bytes;
  int rc = cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
  return rc == PA_OK ? cuda_status(cudaStreamSynchronize(c->stream)) : rc;
}

// Records that everything issued for step t on the run's stream is done (entry t & 3).
void record_step_done(pa_ctx* c, int t) {
  const int i = t & 3;
  c->step_ev_t[i] = -1;
  if (!c->step_ev[i] && cudaEventCreateWithFlags(&c->step_ev[i], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    c->step_ev[i] = nullptr;
    return;
  }
  if (cudaEventRecord(c->step_ev[i], c->stream) == cudaSuccess)
    c->step_ev_t[i] = t;
  else
    cudaGetLastError();
}

// The stream to read step t's results on, once they are complete: the read stream
// waiting for the earliest recorded step u >= t, or, with no such record, the run's
// stream after a full synchronisation.
int read_stream_for(pa_ctx* c, int t, cudaStream_t* out) {
  int best = -1;
  for (int i = 0; i < 4; ++i)
    if (c->step_ev_t[i] >= t && (best < 0 || c->step_ev_t[i] < c->step_ev_t[best])) best = i;
  int prio = 0;
  if (best >= 0 && !c->rd &&
      (cudaStreamGetPriority(c->stream, &prio) != cudaSuccess ||
       cudaStreamCreateWithPriority(&c->rd, cudaStreamNonBlocking, prio) != cudaSuccess)) {
    cudaGetLastError();
    c->rd = nullptr;
  }
  if (best < 0 || !c->rd) {
    *out = c->stream;
    return cuda_status(cudaStreamSynchronize(c->stream));
  }
  *out = c->rd;
  return cuda_status(cudaStreamWaitEvent(c->rd, c->step_ev[best], 0));
}

int copy_d2h_on(pa_ctx* c, cudaStream_t st, void* dst, const void* src, size_t bytes) {
  c->stats.d2h_bytes += (int64_t)bytes;
  int rc = cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
  return rc == PA_OK ? cuda_status(cudaStreamSynchronize(st)) : rc;
}

int copy_h2d(pa_ctx* c, void* dst, const void* src, size_t bytes) {
  c->stats.h2d_bytes += (int64_t)bytes;
  int rc = cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
  return rc == PA_OK ? cuda_status(cudaStreamSynchronize(c->stream)) : rc;
}

// Stream-ordered host-to-device copy; the caller keeps src alive until the stream
// has been synchronised.
int copy_async(pa_ctx* c, void* dst, const void* src, size_t bytes) {
  c->stats.h2d_bytes += (int64_t)bytes;
  return cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
}

cudaEvent_t next_event(pa_ctx* c) {
  if (c->events_used == c->events.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->events.push_back(e);
  }
  return c->events[c->events_used++];
}

// Records CUDA events on the run's stream around one phase when timing is on.
// NVTX range for profilers (no cost unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

const char* const kPhaseNames[PA_N_PHASES] = {"reweight", "resample", "sweep", "family", "overlap"};

struct PhaseTimer {
  pa_ctx* c;
  int phase;
  cudaEvent_t start = nullptr;
  NvtxRange range;
  PhaseTimer(pa_ctx* ctx, int ph, int launches) : c(ctx), phase(ph), range(kPhaseNames[ph]) {
    c->stats.kernel_launches += launches;
    if (c->timing && (start = next_event(c)) != nullptr) cudaEventRecord(start, c->stream);
  }
  ~PhaseTimer() {
    if (!start) return;
    cudaEvent_t end = next_event(c);
    if (!end) return;
    cudaEventRecord(end, c->stream);
    c->timed.push_back({phase, start, end});
  }
};

constexpr size_t kSlabAlign = 256;

// One buffer of the run: with no slab yet (sizing pass) it only adds the buffer's
// aligned size to the total; afterwards it hands out the next piece of the slab.
template <typename T>
int dalloc(pa_ctx* c, T** p, size_t count) {
  if (count == 0) count = 1;
  const size_t bytes = (sizeof(T) * count + kSlabAlign - 1) / kSlabAlign * kSlabAlign;
  if (!c->slab) {
    c->slab_bytes += bytes;
    *p = nullptr;
    return PA_OK;
  }
  if (c->slab_used + bytes > c->slab_bytes) return PA_ERR_NOMEM;  // not laid out in the sizing pass
  *p = reinterpret_cast<T*>(c->slab + c->slab_used);
  c->slab_used += bytes;
  return PA_OK;
}

void make_key(uint64_t seed, uint32_t purpose, uint32_t pop, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32) | (purpose << 28) | (pop << 24);
}

// Metropolis thresholds floor(2^32 exp(-beta dE)), dE = 4, 8, 12, clamped to 2^32 - 1.
void metropolis_thresholds(double beta, uint32_t thr[3]) {
  for (int m = 1; m <= 3; ++m) {
    double p = std::exp(-(beta * (double)(4 * m)));
    double v = std::floor(std::ldexp(p, 32));
    if (v > 4294967295.0) v = 4294967295.0;
    thr[m - 1] = (uint32_t)v;
  }
}

// ---- Gaussian couplings (§II.A), host side: Box-Muller from Philox words at
// counter (n, 1, 0, 0) of the couplings stream, clamped to [-5, 5], fixed point
// Jq = round(J 2^20).  The tables below are what the device needs per step.

void host_philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = (uint32_t)p1;
    c[2] = n2;
    c[3] = (uint32_t)p0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

int32_t fixed_coupling(double g) {
  g = std::min(5.0, std::max(-5.0, g));
  return (int32_t)std::llround(g * 1048576.0);
}

void gauss_couplings(int L, uint64_t seed, std::vector<int32_t>& Jq) {
  const int N = L * L * L;
  Jq.assign((size_t)3 * N, 0);
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffu);
  const uint32_t k1 = (uint32_t)(seed >> 32) | ((uint32_t)pa::kCouplings << 28);
  for (int n = 0; n < N; ++n) {
    uint32_t w[4] = {(uint32_t)n, 1u, 0u, 0u};
    host_philox(w, k0, k1);
    const double u1 = ((double)w[0] + 0.5) * 0x1p-32, u2 = ((double)w[1] + 0.5) * 0x1p-32;
    const double u3 = ((double)w[2] + 0.5) * 0x1p-32, u4 = ((double)w[3] + 0.5) * 0x1p-32;
    const double ra = std::sqrt(-2.0 * std::log(u1)), rb = std::sqrt(-2.0 * std::log(u3));
    const double ta = (2.0 * M_PI) * u2, tb = (2.0 * M_PI) * u4;
    Jq[(size_t)3 * n + 0] = fixed_coupling(ra * std::cos(ta));
    Jq[(size_t)3 * n + 1] = fixed_coupling(ra * std::sin(ta));
    Jq[(size_t)3 * n + 2] = fixed_coupling(rb * std::cos(tb));
  }
}

// Acceptance tables of one step: site n, pattern b of its bonds x+1, x-1, y+1,
// y-1, z+1, z-1 (bit k set: bond k antiparallel), dE = 2 sum_k J_k (1 - 2 b_k):
// the flip's Metropolis threshold, 0xFFFFFFFF for dE <= 0 (always taken), else
// min(floor(2^32 exp(-beta dE 2^-20)), 2^32 - 2) in double precision.
void gauss_site_tables_range(const std::vector<int32_t>& Jq, int L, double beta, uint32_t* out, int n0, int n1) {
  for (int n = n0; n < n1; ++n) {
    const int x = n % L, y = (n / L) % L, z = n / (L * L);
    const int xm = (x == 0 ? L - 1 : x - 1) + L * (y + L * z);
    const int ym = x + L * ((y == 0 ? L - 1 : y - 1) + L * z);
    const int zm = x + L * (y + L * (z == 0 ? L - 1 : z - 1));
    const int64_t bond[6] = {Jq[(size_t)3 * n + 0], Jq[(size_t)3 * xm + 0], Jq[(size_t)3 * n + 1],
                             Jq[(size_t)3 * ym + 1], Jq[(size_t)3 * n + 2], Jq[(size_t)3 * zm + 2]};
    for (int b = 0; b < pa::kGPatterns; ++b) {
      int64_t dE = 0;  // flipping s_n: +2J for a parallel neighbour, -2J for an antiparallel one
      for (int k = 0; k < 6; ++k) dE += bond[k] * (((b >> k) & 1) ? -1 : 1);
      dE *= 2;
      uint32_t thr = 0xFFFFFFFFu;
      if (dE > 0) {
        double v = std::floor(std::exp(-(beta * ((double)dE * 0x1p-20))) * 4294967296.0);
        if (v > 4294967294.0) v = 4294967294.0;
        thr = (uint32_t)v;
      }
      out[(size_t)n * pa::kGPatterns + b] = thr;
    }
  }
}

// The site tables of all N sites; a large lattice's sites are split over a few
// host threads (each entry is a function of its site alone, so the table is the same).
void gauss_site_tables(const std::vector<int32_t>& Jq, int L, double beta, uint32_t* out) {
  const int N = L * L * L;
  const int n_thr = N < 512 ? 1 : (int)std::min<unsigned>(8u, std::max(1u, std::thread::hardware_concurrency()));
  if (n_thr == 1) {
    gauss_site_tables_range(Jq, L, beta, out, 0, N);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve((size_t)n_thr);
  const int per = (N + n_thr - 1) / n_thr;
  for (int k = 1; k < n_thr && k * per < N; ++k) {
    const int a = k * per, b = std::min(N, (k + 1) * per);
    try {
      pool.emplace_back(gauss_site_tables_range, std::cref(Jq), L, beta, out, a, b);
    } catch (const std::system_error&) {  // no thread to be had: this range here
      gauss_site_tables_range(Jq, L, beta, out, a, b);
    }
  }
  gauss_site_tables_range(Jq, L, beta, out, 0, std::min(N, per));
  for (std::thread& th : pool) th.join();
}

// Uploads the adaptive Gaussian step's site tables for beta, built into a pinned
// buffer and copied without a wait (plain copy where pinned memory is not had).
// The previous step's copy from that buffer is done: the bisection that chose beta
// synchronised the stream.
int upload_site_tables(pa_ctx* c, double beta) {
  const size_t n = (size_t)c->g.N * pa::kGPatterns;
  if (!c->gtab_host) {
    void* h = nullptr;
    if (cudaMallocHost(&h, sizeof(uint32_t) * n) == cudaSuccess)
      c->gtab_host = static_cast<uint32_t*>(h);
    else
      cudaGetLastError();
  }
  if (!c->gtab_host) {
    std::vector<uint32_t> tab(n);
    gauss_site_tables(c->Jq_host, c->g.L, beta, tab.data());
    return copy_h2d(c, c->gtab, tab.data(), sizeof(uint32_t) * n);
  }
  gauss_site_tables(c->Jq_host, c->g.L, beta, c->gtab_host);
  return copy_async(c, c->gtab, c->gtab_host, sizeof(uint32_t) * n);
}

// Weight tables of one step: T0[m] = exp(-dbeta m 2^-20), T1[m] for m 2^12,
// T2[m] for m 2^24 (8192 entries).
void gauss_weight_tables(double dbeta, double* T) {
  for (int m = 0; m < 4096; ++m) T[m] = std::exp(-(dbeta * ((double)m * 0x1p-20)));
  for (int m = 0; m < 4096; ++m) T[4096 + m] = std::exp(-(dbeta * ((double)((int64_t)m << 12) * 0x1p-20)));
  for (int m = 0; m < 8192; ++m) T[8192 + m] = std::exp(-(dbeta * ((double)((int64_t)m << 24) * 0x1p-20)));
}

uint64_t bits_of(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
}

// Host table w[j] = exp(-(dbeta * 2j)), j = 0..3N: the Boltzmann weight ratio of
// a temperature move between a level and the lowest occupied one.
std::vector<double> host_weights(int n_levels, double dbeta) {
  std::vector<double> w((size_t)n_levels);
  for (int j = 0; j < n_levels; ++j) w[(size_t)j] = std::exp(-(dbeta * (double)(2 * j)));
  return w;
}

// Explicit schedules of many runs share their increments (a linear schedule has a
// handful of distinct ones), so their tables are computed once per process.
std::shared_ptr<const std::vector<double>> cached_weights(int n_levels, double dbeta) {
  static std::mutex mu;
  static std::map<std::pair<int, uint64_t>, std::shared_ptr<const std::vector<double>>> cache;
  const std::pair<int, uint64_t> key(n_levels, bits_of(dbeta));
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  if (cache.size() >= 1024) cache.clear();  // bounded: at most 1024 tables of <= 12289 doubles
  auto w = std::make_shared<const std::vector<double>>(host_weights(n_levels, dbeta));
  cache.emplace(key, w);
  return w;
}

// Device weight table of step t.  Explicit schedules upload one table per
// distinct dbeta at creation; the adaptive schedule rewrites one buffer after
// the host has synchronised to choose dbeta (so no kernel still reads it).
int weight_table(pa_ctx* c, double dbeta, const double** out) {
  if (!c->adaptive) {  // every table of an explicit schedule was uploaded at creation
    auto it = c->wtables.find(bits_of(dbeta));
    if (it == c->wtables.end()) return PA_ERR_INVALID;
    *out = it->second;
    return PA_OK;
  }
  // The reweighting reads w[k - kmin] at the occupied levels k only; with one
  // population they span occ_span + 1 entries (choose_dbeta found them), and the
  // entries past those are zeros instead of exponentials.
  const int n = c->g.n_levels;
  const int used = c->g.n_pop == 1 && c->occ_span >= 0 ? std::min(n, c->occ_span + 1) : n;
  std::vector<double> w((size_t)n, 0.0);
  for (int j = 0; j < used; ++j) w[(size_t)j] = std::exp(-(dbeta * (double)(2 * j)));
  const size_t bytes = sizeof(double) * w.size();
  if (!c->wadapt_host) {  // pinned, so the upload need not wait (first use; else plain copies)
    void* h = nullptr;
    if (cudaMallocHost(&h, bytes) == cudaSuccess)
      c->wadapt_host = static_cast<double*>(h);
    else
      cudaGetLastError();
  }
  if (!c->wadapt_host) {
    const int rc = copy_h2d(c, c->wadapt, w.data(), bytes);
    if (rc != PA_OK) return rc;
  } else {
    // the previous step's upload from this buffer is done: choose_dbeta synchronised the
    // stream before this step's table was built
    std::memcpy(c->wadapt_host, w.data(), bytes);
    const int rc = copy_async(c, c->wadapt, c->wadapt_host, bytes);
    if (rc != PA_OK) return rc;
  }
  *out = c->wadapt;
  return PA_OK;
}

// Expected culling fraction (1/R) sum_k c(k) (1 - tau_k)_+ of a move by dbeta
// from level histogram c (occupied levels only; empty ones add exact zeros).  The
// weights of the first sum are kept in w for the second (each is one exp of the
// same argument either way, so the result does not change).
double culling_fraction(const std::vector<int32_t>& occ, const std::vector<uint32_t>& c, int64_t R, double dbeta,
                        std::vector<double>& w) {
  const int kmin = occ[0];
  w.resize(occ.size());
  double S = 0.0;
  for (size_t i = 0; i < occ.size(); ++i) {
    w[i] = std::exp(-(dbeta * (double)(2 * (occ[i] - kmin))));
    S = S + (double)c[(size_t)occ[i]] * w[i];
  }
  double eps = 0.0;
  for (size_t i = 0; i < occ.size(); ++i) {
    const double tau = ((double)R * w[i]) / S;
    if (tau < 1.0) eps = eps + (double)c[(size_t)occ[i]] * (1.0 - tau);
  }
  return eps / (double)R;
}

// Adaptive step (§IV.B): the largest dbeta in (0, beta_max - beta] whose expected
// culling fraction does not exceed the target, by 64 bisection halvings;
// population 0 decides.
int choose_dbeta(pa_ctx* c, double* dbeta) {
  const int n = c->g.n_levels;
  std::vector<uint32_t> h((size_t)n);
  int rc = cuda_status(cudaStreamSynchronize(c->stream));
  if (rc == PA_OK) rc = copy_d2h(c, h.data(), c->pops[0].hist + (size_t)(c->t) * n, sizeof(uint32_t) * n);
  if (rc != PA_OK) return rc;
  std::vector<int32_t> occ;
  for (int k = 0; k < n; ++k)
    if (h[(size_t)k] > 0) occ.push_back(k);
  if (occ.empty()) return PA_ERR_EXTINCT;
  c->occ_span = occ.back() - occ.front();
  const double prev = c->betas[(size_t)c->t];
  const double rem = c->cfg.beta_max - prev;
  const double target = c->cfg.eps_target;
  std::vector<double> w;
  if (culling_fraction(occ, h, c->cfg.R, rem, w) <= target) {
    *dbeta = rem;
    return PA_OK;
  }
  double lo = 0.0, hi = rem;
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi);
    // a midpoint equal to hi (rejected) or to lo > 0 (accepted) is decided already,
    // and so is every later one: the remaining halvings would change nothing
    if (mid == hi || (mid == lo && lo > 0.0)) break;
    if (culling_fraction(occ, h, c->cfg.R, mid, w) <= target)
      lo = mid;
    else
      hi = mid;
  }
  *dbeta = lo > 0.0 ? lo : hi;
  return PA_OK;
}

// Adaptive step for Gaussian couplings: the same bisection, with the culling
// fraction of each trial computed on the device from that trial's weight tables
// (the definitions the resampling uses), population 0 deciding.
// Observables of step t of a +-1 population (pa_obs) from its step records and level
// histograms of steps 0..t (rec, hall: (t + 1) x n_levels) and, with two
// populations, population 0's record of step t (r0, else null): Eqs. (Q), (betaF),
// (g0), the family statistics and the overlap counts.
void pm1_observables(const RunGeom& g, const std::vector<double>& betas, const StepRec* rec, const uint32_t* h,
                     int t, const StepRec* r0, pa_obs* out) {
  const int N = g.N;
  // free energy, Eq. (betaF), and the lowest energy over steps 0..t: the lowest
  // occupied level of step u < t is the one the reweighting of step u + 1 recorded
  double lnQ_sum = 0.0, lnQ = 0.0;
  int32_t E0 = 3 * N + 1;
  for (int u = 1; u <= t; ++u) {
    const StepRec& r = rec[(size_t)u];
    const double db = betas[(size_t)u] - betas[(size_t)u - 1];
    const int32_t Emin_prev = 2 * r.kmin_prev - 3 * N;
    lnQ = std::log(r.S_prime / (double)r.R_prev) - db * (double)Emin_prev;
    lnQ_sum = lnQ_sum + lnQ;
    E0 = std::min(E0, Emin_prev);
  }
  pa_obs o{};
  const StepRec& r = rec[(size_t)t];
  o.t = t;
  o.beta = betas[(size_t)t];
  o.dbeta = t > 0 ? betas[(size_t)t] - betas[(size_t)t - 1] : 0.0;
  o.R_tilde = r.R_tilde;
  int64_t sE = 0, sE2 = 0;
  int32_t Emin = 3 * N + 1;
  for (int k = 0; k < g.n_levels; ++k) {
    if (!h[k]) continue;
    const int64_t E = 2 * k - 3 * N;
    sE += (int64_t)h[k] * E;
    sE2 += (int64_t)h[k] * E * E;
    Emin = std::min<int32_t>(Emin, (int32_t)E);
  }
  o.sum_E = sE;
  o.sum_E2 = sE2;
  o.E_min = Emin;
  E0 = std::min(E0, Emin);
  o.mean_E = (double)sE / (double)o.R_tilde;
  o.var_E = (double)sE2 / (double)o.R_tilde - o.mean_E * o.mean_E;
  o.kmin_prev = t > 0 ? r.kmin_prev : 0;
  o.S_prime = t > 0 ? r.S_prime : 0.0;
  o.lnQ = t > 0 ? lnQ : 0.0;
  o.minus_beta_F = (double)N * std::log(2.0) + lnQ_sum;
  o.eps_expected = t > 0 ? r.eps_expected : 0.0;
  o.culled = t > 0 ? r.culled : 0;
  o.sum_eta2 = (int64_t)r.sum_eta2;
  o.n_families = (int64_t)r.n_families;
  o.rho_t = (double)o.sum_eta2 / (double)o.R_tilde;
  o.S_f = -nu_ln_nu(r);
  o.rho_s = (double)o.R_tilde / std::exp(o.S_f);
  o.E0 = E0;
  o.g0_tilde = (double)h[(E0 + 3 * N) / 2] / (double)o.R_tilde;
  o.g0_bar = 2.0 * std::exp(-(o.beta * (double)E0) - o.minus_beta_F);
  if (r0) {
    o.q_pairs = (int64_t)r0->q_pairs;
    o.q_abs_le_02 = (int64_t)r0->q_small;
    o.I02 = o.q_pairs > 0 ? (double)o.q_abs_le_02 / (double)o.q_pairs : 0.0;
  }
  *out = o;
}

int launch_rc(int e) { return e == 0 ? PA_OK : PA_ERR_CUDA; }

// Adaptive step with Gaussian couplings (§IV.B), as for +-1 couplings: the largest
// dbeta in (0, beta_max - beta] whose culling fraction (population 0, the
// resampling's own weights and sums) does not exceed the target, by 64 bisection
// halvings.  The halvings run on the device in one cooperative launch
// (launch_g_bisect_fused; one launch per halving where that is not possible) with
// no host wait between them; the host reads the first trial (the whole remaining
// range) and the final interval.
int choose_dbeta_gauss(pa_ctx* c, double* dbeta) {
  const int t = c->t + 1;
  const double rem = c->cfg.beta_max - c->betas[(size_t)c->t];
  const double target = c->cfg.eps_target;
  double b[4] = {0.0, rem, rem, 0.0};
  int rc = copy_h2d(c, c->gbis, b, sizeof b);
  if (rc == PA_OK) rc = launch_rc(pa::launch_g_tables(c->gbis + 2, 0.0, c->gw, c->stream));
  if (rc == PA_OK) rc = launch_rc(pa::launch_g_eps_trial(c->g, c->pops, t, c->gw, c->stream));
  double e = 0.0;
  if (rc == PA_OK) rc = copy_d2h(c, &e, &c->pops[0].rec[t].eps_expected, sizeof(double));
  if (rc != PA_OK) return rc;
  if (e <= target) {
    *dbeta = rem;
    return PA_OK;
  }
  b[2] = 0.5 * (b[0] + b[1]);
  rc = copy_h2d(c, c->gbis, b, sizeof b);
  if (c->gbis_blocks < 0) c->gbis_blocks = pa::g_bisect_blocks(c->g);
  if (rc == PA_OK && c->gbis_blocks > 0)
    rc = launch_rc(pa::launch_g_bisect_fused(c->g, c->pops, t, c->gbt, c->gbt + 3 * (size_t)pa::kGTableWeights,
                                             c->gbar, c->gbis, target, 64, c->gbis_blocks, c->gbis_withheld,
                                             c->stream));
  else if (rc == PA_OK)
    rc = launch_rc(pa::launch_g_bisect(c->g, c->pops, t, c->gw, c->gbis, target, 64, c->stream));
  if (rc == PA_OK) rc = copy_d2h(c, b, c->gbis, sizeof b);
  if (rc != PA_OK) return rc;
  if (b[3] < 0.0) return PA_ERR_TIMEOUT;
  *dbeta = b[0] > 0.0 ? b[0] : b[1];
  return PA_OK;
}

int check_device_status(pa_ctx* c) {
  int32_t flags = 0;
  int rc = cuda_status(cudaStreamSynchronize(c->stream));
  if (rc == PA_OK) rc = copy_d2h(c, &flags, c->status, sizeof flags);
  if (rc != PA_OK) return rc;
  if (flags & pa::kFlagCapacity) return PA_ERR_CAPACITY;
  if (flags & pa::kFlagExtinct) return PA_ERR_EXTINCT;
  if (flags & pa::kFlagTimeout) return PA_ERR_TIMEOUT;
  return PA_OK;
}

int fail(pa_ctx* c, int rc) {
  if (rc != PA_OK && c->error == PA_OK) c->error = rc;
  return rc;
}




// Measurement kernels common to every step: families (and overlap).
int measure(pa_ctx* c, int t) {
  int rc = PA_OK;
  if (c->model == PA_MODEL_GAUSS) {
    PhaseTimer pt(c, PA_PHASE_FAMILY, 3);
    rc = launch_rc(pa::launch_g_measure(c->g, c->pops, c->cur, t, c->qlhist, c->stream));
  }
  // the +-1 shared-memory sweep adds the family statistics of steps t >= 1 itself
  const bool in_sweep = c->model == PA_MODEL_PM1 && t > 0 && pa::sweep_supported(c->g.L);
  if (rc == PA_OK && !in_sweep) {
    PhaseTimer pt(c, PA_PHASE_FAMILY, 1);
    rc = launch_rc(pa::launch_families(c->g, c->pops, c->cur, t, c->stream));
  }
  if (rc == PA_OK && c->g.n_pop == 2) {
    PhaseTimer pt(c, PA_PHASE_OVERLAP, 1);
    rc = launch_rc(pa::launch_overlap(c->g, c->pops, c->cur, t, c->qhist, c->stream));
  }
  return rc;
}

void destroy(pa_ctx* c) {
  if (!c) return;
  if (c->slab) cudaFreeAsync(c->slab, c->stream);
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  for (cudaEvent_t e : c->step_ev)
    if (e) cudaEventDestroy(e);
  if (c->rd) cudaStreamDestroy(c->rd);
  if (c->wadapt_host) cudaFreeHost(c->wadapt_host);
  if (c->gtab_host) cudaFreeHost(c->gtab_host);
  delete c;
}

}  // namespace

// ---------------------------------------------------------------- checkpoint / restore
//
// Layout of a checkpoint (host byte order): CkptHeader, the schedule (betas and
// sweeps of all n_temps steps), then per population: step records and level
// histograms of steps 0..t, the spins of the current population (site-major,
// N rows of R~ bytes), its labels and levels, the copy numbers of the last
// resampling (R~_{t-1} entries), the parent map (R~ entries) and the family-size
// histogram (R~ + 1 entries); then the overlap histograms of steps 0..t.  A run
// with Gaussian couplings stores, per population, the step records and Gaussian
// step records of steps 0..t, the spins, labels, energies (int64, fixed point),
// copy numbers, parents and family-size histogram, then the overlap and
// link-overlap histograms of steps 0..t.

namespace {

struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int32_t L, n_pop, q_bins, n_temps;
  int64_t R, R_cap;
  uint64_t disorder_seed, run_seed;
  double eps_target, beta_max;
  int32_t t, done, adaptive, n_sweeps;
  int32_t R_tilde[2], R_prev[2];
  int32_t model, pad;
  uint64_t total_bytes;
};
constexpr char kCkptMagic[8] = {'P', 'A', 'C', 'K', 'P', 'T', '0', '1'};
// Version 4: the Gaussian model's Metropolis uniforms come from 16-bit halves (a
// version 3 checkpoint would resume on other random numbers than it started with).
constexpr uint32_t kCkptVersion = 4;

size_t ckpt_bytes(const RunGeom& g, int model, int t, int n_temps, const int32_t* Rt, const int32_t* Rp) {
  size_t b = sizeof(CkptHeader) + (size_t)n_temps * (sizeof(double) + sizeof(int32_t));
  const bool gauss = model == PA_MODEL_GAUSS;
  for (int p = 0; p < g.n_pop; ++p) {
    b += (size_t)(t + 1) * (sizeof(StepRec) + (gauss ? sizeof(pa::GRec) : sizeof(uint32_t) * (size_t)g.n_levels));
    b += (size_t)g.N * (size_t)Rt[p];  // spins
    // labels, levels or energies, parents, counts, family-size histogram
    b += sizeof(int32_t) * ((size_t)Rt[p] * 2 + (size_t)Rp[p] + (size_t)Rt[p] + 1);
    b += (gauss ? sizeof(int64_t) : sizeof(int32_t)) * (size_t)Rt[p];
  }
  b += (gauss ? 2 : 1) * sizeof(unsigned long long) * (size_t)(t + 1) * (size_t)g.q_bins;
  return b;
}

// Population capacity of a configuration (R_cap = 0: R + 10 sqrt(R) + 1024).
int64_t capacity_of(const pa_config* cfg) {
  return cfg->R_cap ? cfg->R_cap : cfg->R + 10 * (int64_t)std::ceil(std::sqrt((double)cfg->R)) + 1024;
}

// The distinct increments beta_t - beta_{t-1} of an explicit schedule, in order of
// first use (one Boltzmann weight table each).
std::vector<double> distinct_dbetas(const std::vector<double>& betas) {
  std::vector<double> out;
  std::map<uint64_t, int> seen;
  for (size_t t = 1; t < betas.size(); ++t) {
    const double d = betas[t] - betas[t - 1];
    if (seen.emplace(bits_of(d), 0).second) out.push_back(d);
  }
  return out;
}

// Copies the configuration and schedule into c and sets up the run's geometry
// (no device call; the sweep shape is left at the default).
void init_run(pa_ctx* c, const pa_config* cfg, int64_t R_cap) {
  c->cfg = *cfg;
  c->cfg.R_cap = R_cap;
  c->adaptive = cfg->betas == nullptr;
  c->betas.assign((size_t)cfg->n_temps, 0.0);
  c->sweeps.assign((size_t)cfg->n_temps, cfg->n_sweeps);
  for (int t = 0; t < cfg->n_temps; ++t) {
    if (cfg->betas) c->betas[(size_t)t] = cfg->betas[t];
    if (cfg->sweeps_per_step) c->sweeps[(size_t)t] = cfg->sweeps_per_step[t];
  }
  c->cfg.betas = nullptr;
  c->cfg.sweeps_per_step = nullptr;
  RunGeom& g = c->g;
  g.L = cfg->L;
  g.N = cfg->L * cfg->L * cfg->L;
  g.n_levels = 3 * g.N + 1;
  g.pitch = ((R_cap + 1023) / 1024) * 1024;  // a whole number of sweep tiles (<= 1024 replicas)
  g.R = (int32_t)cfg->R;
  g.R_cap = (int32_t)R_cap;
  g.n_pop = cfg->n_pop;
  g.q_bins = cfg->q_bins;
  g.n_count_blocks = (int32_t)((R_cap + pa::kSlotsPerCountBlock - 1) / pa::kSlotsPerCountBlock);
  // K distinct family sizes add up to at least K (K + 1) / 2 <= R~, so K <= floor(sqrt(2 R_cap))
  int64_t k = (int64_t)std::sqrt(2.0 * (double)R_cap);
  while ((k + 1) * (k + 1) <= 2 * R_cap) ++k;
  while (k * k > 2 * R_cap) --k;
  g.n_fsizes = (int32_t)k + 2;
  g.sweep_shape = 0;
  g.tail_shape = -1;
  g.tail_from = 0;
  g.model = cfg->model;
  g.slot_base = 0;
  g.n_init = (int32_t)cfg->R;
  g.shard = 0;
  g.n_chunks = (int32_t)((R_cap + pa::kChunk - 1) / pa::kChunk);
  g.n_measure_blocks = (int32_t)((R_cap + 4095) / 4096);
  c->model = cfg->model;
}

// The run's device buffers in one fixed order: sizes only while c has no slab,
// else carved from it (the two passes lay out the same buffers).
int layout_buffers(pa_ctx* c) {
  const RunGeom& g = c->g;
  const size_t T = c->betas.size();
  int rc = PA_OK;
  rc = rc ? rc : dalloc(c, &c->J, (size_t)3 * g.N);
  rc = rc ? rc : dalloc(c, &c->jtab, (size_t)4 * g.N);
  rc = rc ? rc : dalloc(c, &c->status, 1);
  rc = rc ? rc : dalloc(c, &c->qhist, T * (size_t)g.q_bins);
  for (int p = 0; p < g.n_pop && rc == PA_OK; ++p) {
    PopDev& P = c->pops[p];
    for (int b = 0; b < 2 && rc == PA_OK; ++b) {
      rc = dalloc(c, &P.spins[b], (size_t)g.N * (size_t)g.pitch);
      rc = rc ? rc : dalloc(c, &P.labels[b], (size_t)g.pitch);
    }
    rc = rc ? rc : dalloc(c, &P.levels, (size_t)g.pitch);
    rc = rc ? rc : dalloc(c, &P.counts, (size_t)g.pitch);
    rc = rc ? rc : dalloc(c, &P.parents, (size_t)g.pitch);
    rc = rc ? rc : dalloc(c, &P.blocksums, (size_t)g.n_count_blocks);
    rc = rc ? rc : dalloc(c, &P.tiles, (size_t)g.n_count_blocks);
    rc = rc ? rc : dalloc(c, &P.ticket, (size_t)1);
    rc = rc ? rc : dalloc(c, &P.hist, T * (size_t)g.n_levels);
    rc = rc ? rc : dalloc(c, &P.fl, (size_t)g.n_levels);
    rc = rc ? rc : dalloc(c, &P.thr, (size_t)g.n_levels);
    rc = rc ? rc : dalloc(c, &P.mhist, (size_t)g.R_cap + 1);
    rc = rc ? rc : dalloc(c, &P.fhist, (size_t)g.R_cap + 1);
    rc = rc ? rc : dalloc(c, &P.fsizes, (size_t)g.n_fsizes);
    rc = rc ? rc : dalloc(c, &P.fcount, (size_t)2);
    rc = rc ? rc : dalloc(c, &P.rec, T);
    if (g.model == PA_MODEL_GAUSS) {
      rc = rc ? rc : dalloc(c, &P.E64, (size_t)g.pitch);
      rc = rc ? rc : dalloc(c, &P.w, (size_t)g.R_cap);
      rc = rc ? rc : dalloc(c, &P.part, (size_t)pa::tree_sum_scratch(g.n_chunks));
      rc = rc ? rc : dalloc(c, &P.gfl, (size_t)g.R_cap);
      rc = rc ? rc : dalloc(c, &P.gthr, (size_t)g.R_cap);
      rc = rc ? rc : dalloc(c, &P.e2part, (size_t)2 * g.n_measure_blocks);
      rc = rc ? rc : dalloc(c, &P.grec, T);
    }
  }
  if (g.model == PA_MODEL_GAUSS) {
    rc = rc ? rc : dalloc(c, &c->Jq, (size_t)3 * g.N);
    const size_t slots = c->adaptive ? 1 : T;  // adaptive: this step's tables, rebuilt every step
    rc = rc ? rc : dalloc(c, &c->gtab, slots * (size_t)g.N * pa::kGPatterns);
    rc = rc ? rc : dalloc(c, &c->gw, slots * (size_t)pa::kGTableWeights);
    rc = rc ? rc : dalloc(c, &c->qlhist, T * (size_t)g.q_bins);
    if (c->adaptive) {
      rc = rc ? rc : dalloc(c, &c->gbis, (size_t)4);
      rc = rc ? rc : dalloc(c, &c->gbt, (size_t)3 * pa::kGTableWeights + (size_t)g.n_chunks);
      rc = rc ? rc : dalloc(c, &c->gbar, (size_t)8);
    }
  } else if (c->adaptive) {
    rc = rc ? rc : dalloc(c, &c->wadapt, (size_t)g.n_levels);
  } else {  // one Boltzmann weight table per distinct increment
    const std::vector<double> d = distinct_dbetas(c->betas);
    double* all = nullptr;
    rc = rc ? rc : dalloc(c, &all, d.size() * (size_t)g.n_levels);
    if (rc == PA_OK && all)
      for (size_t i = 0; i < d.size(); ++i) c->wtables[bits_of(d[i])] = all + i * (size_t)g.n_levels;
  }
  return rc;
}

}  // namespace

namespace pa {
// Runs overlapped with many others (pa_batch, pa_server) keep the device's chosen
// sweep shape: their tiles need not fill the GPU by themselves.
void use_chosen_shape(pa_ctx* c) {
  int dev = 0;
  if (c && sweep_supported(c->g.L) && current_device(&dev) == PA_OK) c->g.sweep_shape = g_sweep_choice[dev][c->g.L].load();
  if (c) c->g.tail_shape = -1;  // runs among many: other runs fill the SMs a last wave leaves idle
}

int exception_status() noexcept {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    return PA_ERR_NOMEM;
  } catch (...) {
    return PA_ERR_INVALID;
  }
}
}  // namespace pa

namespace {

template <typename T>
T read_at(const char* p, size_t i) {
  T v;
  std::memcpy(&v, p + i * sizeof(T), sizeof(T));
  return v;
}

// Checks the population part of a checkpoint on the host, before any of it
// reaches the device: every value a kernel later uses as an index or a size must
// be in range and consistent.  Step records chain (each step's previous size is
// the last step's size, sizes within the capacity, the lowest level in range),
// level histograms add up to their population, spins are +-1, labels ascend and
// stay below R, levels lie in range and match the last histogram, copy numbers
// are non-negative and add up to the population, parents ascend within the old
// population, family-size counts are non-negative and cover the population.  `in` points just past the
// schedule; the size of the whole buffer has been checked already.
bool ckpt_payload_ok(const RunGeom& g, bool gauss, int t, int64_t R, const CkptHeader& h, const char* in) {
  const int64_t max_abs_E = 3 * (int64_t)g.N * 5 * ((int64_t)1 << 20);  // Gaussian couplings are clamped to 5
  for (int p = 0; p < g.n_pop; ++p) {
    const int64_t Rt = h.R_tilde[p], Rp = h.R_prev[p];
    std::vector<StepRec> rec((size_t)t + 1);
    std::memcpy(rec.data(), in, sizeof(StepRec) * rec.size());
    in += sizeof(StepRec) * rec.size();
    for (int u = 0; u <= t; ++u) {
      const StepRec& r = rec[(size_t)u];
      if (r.R_tilde < 1 || r.R_tilde > g.R_cap) return false;
      if (u > 0 && (r.R_prev != rec[(size_t)u - 1].R_tilde || r.S_t < 0 || r.culled < 0 || r.culled > r.R_prev))
        return false;
      if (u > 0 && !gauss && (r.kmin_prev < 0 || r.kmin_prev >= g.n_levels)) return false;
    }
    if (rec[0].R_tilde != R || rec[(size_t)t].R_tilde != Rt || (t > 0 ? rec[(size_t)t].R_prev : 0) != Rp)
      return false;
    long long E_min = 0;
    std::vector<int64_t> last_hist;
    if (gauss) {
      E_min = read_at<pa::GRec>(in, (size_t)t).E_min;
      in += sizeof(pa::GRec) * ((size_t)t + 1);
    } else {
      for (int u = 0; u <= t; ++u) {
        int64_t sum = 0;
        for (int k = 0; k < g.n_levels; ++k) sum += read_at<uint32_t>(in, (size_t)u * g.n_levels + k);
        if (sum != rec[(size_t)u].R_tilde) return false;
      }
      last_hist.resize((size_t)g.n_levels);
      for (int k = 0; k < g.n_levels; ++k)
        last_hist[(size_t)k] = read_at<uint32_t>(in, (size_t)t * g.n_levels + k);
      in += sizeof(uint32_t) * ((size_t)t + 1) * (size_t)g.n_levels;
    }
    const size_t n_spins = (size_t)g.N * (size_t)Rt;
    for (size_t i = 0; i < n_spins; ++i) {
      const uint8_t b = (uint8_t)in[i];
      if (b != 0x01 && b != 0xFF) return false;
    }
    in += n_spins;
    for (int64_t j = 0; j < Rt; ++j) {
      const int32_t l = read_at<int32_t>(in, (size_t)j);
      if (l < 0 || l >= R || (j > 0 && l < read_at<int32_t>(in, (size_t)j - 1))) return false;
    }
    in += sizeof(int32_t) * (size_t)Rt;
    if (gauss) {
      long long lo = 0;
      for (int64_t j = 0; j < Rt; ++j) {
        const long long e = read_at<int64_t>(in, (size_t)j);
        if (e < -max_abs_E || e > max_abs_E) return false;
        lo = j == 0 ? e : std::min(lo, e);
      }
      if (lo != E_min) return false;
      in += sizeof(int64_t) * (size_t)Rt;
    } else {
      for (int64_t j = 0; j < Rt; ++j) {
        const int32_t k = read_at<int32_t>(in, (size_t)j);
        if (k < 0 || k >= g.n_levels) return false;
        --last_hist[(size_t)k];
      }
      for (int64_t c : last_hist)
        if (c != 0) return false;
      in += sizeof(int32_t) * (size_t)Rt;
    }
    int64_t copies = 0;
    for (int64_t i = 0; i < Rp; ++i) {
      const int32_t n = read_at<int32_t>(in, (size_t)i);
      if (n < 0) return false;
      copies += n;
    }
    if (t > 0 && copies != Rt) return false;
    in += sizeof(int32_t) * (size_t)Rp;
    for (int64_t j = 0; j < Rt; ++j) {
      const int32_t q = read_at<int32_t>(in, (size_t)j);
      if (q < 0 || q >= g.R_cap) return false;
      if (t > 0 && (q >= Rp || (j > 0 && q < read_at<int32_t>(in, (size_t)j - 1)))) return false;
    }
    in += sizeof(int32_t) * (size_t)Rt;
    int64_t members = 0;
    for (int64_t e = 0; e <= Rt; ++e) {
      const int32_t m = read_at<int32_t>(in, (size_t)e);
      if (m < 0) return false;
      members += e * (int64_t)m;
    }
    if (members != Rt) return false;
    in += sizeof(int32_t) * ((size_t)Rt + 1);
  }
  return true;
}

}  // namespace

extern "C" {

const char* pa_strerror(int s) {
  switch (s) {
    case PA_OK: return "ok";
    case PA_DONE: return "schedule complete";
    case PA_ERR_INVALID: return "invalid argument or configuration";
    case PA_ERR_NOMEM: return "out of memory";
    case PA_ERR_CAPACITY: return "population exceeded its capacity R_cap";
    case PA_ERR_TIMEOUT: return "a bounded device wait timed out";
    case PA_ERR_CUDA: return "CUDA runtime error";
    case PA_ERR_STATE: return "call out of order";
    case PA_ERR_EXTINCT: return "population became empty";
    default: return "unknown status";
  }
}

int pa_footprint(const pa_config* cfg, size_t* bytes) try {
  if (!cfg || !bytes || !pa::lattice_supported(cfg->L) || cfg->R < 1 || cfg->n_temps < 1 || cfg->n_pop < 1 ||
      cfg->n_pop > 2 || cfg->model < PA_MODEL_PM1 || cfg->model > PA_MODEL_GAUSS || cfg->q_bins < 0)
    return PA_ERR_INVALID;
  pa_ctx sizing;  // the sizing pass of the buffer layout: no device memory is touched
  init_run(&sizing, cfg, capacity_of(cfg));
  const int rc = layout_buffers(&sizing);
  if (rc != PA_OK) return rc;
  *bytes = sizing.slab_bytes;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

}  // extern "C"

namespace {
struct SharePlacement {
  bool share = false;
  int64_t slot_base = 0, n_init = 0;
};
int create_run_impl(const pa_config* cfg, void* cuda_stream, pa_ctx** out, bool synchronize, const SharePlacement& sp);
}  // namespace

int pa::create_run(const pa_config* cfg, void* cuda_stream, pa_ctx** out, bool synchronize) {
  return create_run_impl(cfg, cuda_stream, out, synchronize, SharePlacement{});
}

int pa::create_run_share(const pa_config* cfg, void* cuda_stream, pa_ctx** out, int64_t slot_base, int64_t n_init) {
  SharePlacement sp;
  sp.share = true;
  sp.slot_base = slot_base;
  sp.n_init = n_init;
  return create_run_impl(cfg, cuda_stream, out, true, sp);
}

namespace {
int create_run_impl(const pa_config* cfg, void* cuda_stream, pa_ctx** out, bool synchronize, const SharePlacement& sp) {
  if (!out) return PA_ERR_INVALID;
  *out = nullptr;
  if (!cfg) return PA_ERR_INVALID;
  const int64_t R_cap = capacity_of(cfg);
  if (!pa::lattice_supported(cfg->L) || cfg->R < 1 || cfg->n_pop < 1 || cfg->n_pop > 2 || cfg->n_temps < 1 ||
      R_cap < cfg->R || R_cap >= ((int64_t)1 << 31) - 4096 || cfg->disorder_seed >= ((uint64_t)1 << 56) ||
      cfg->run_seed >= ((uint64_t)1 << 56) || cfg->q_bins < 3 || cfg->q_bins > 4097 || cfg->n_sweeps < 0)
    return PA_ERR_INVALID;
  if (!cfg->betas && !(cfg->eps_target > 0.0 && cfg->eps_target < 1.0 && cfg->beta_max > 0.0)) return PA_ERR_INVALID;
  if (cfg->model < PA_MODEL_PM1 || cfg->model > PA_MODEL_GAUSS ||
      (cfg->model == PA_MODEL_GAUSS && !pa::sweep_supported(cfg->L)))
    return PA_ERR_INVALID;
  if (cfg->betas) {
    if (cfg->betas[0] != 0.0) return PA_ERR_INVALID;
    for (int t = 1; t < cfg->n_temps; ++t)
      if (!(cfg->betas[t] >= cfg->betas[t - 1])) return PA_ERR_INVALID;
  }
  if (cfg->sweeps_per_step)
    for (int t = 0; t < cfg->n_temps; ++t)
      if (cfg->sweeps_per_step[t] < 0) return PA_ERR_INVALID;

  if (sp.share && (sp.slot_base < 0 || sp.slot_base % 1024 != 0 || sp.n_init < 0 || sp.slot_base + sp.n_init > cfg->R))
    return PA_ERR_INVALID;
  pa_ctx* c = new (std::nothrow) pa_ctx();
  if (!c) return PA_ERR_NOMEM;
  init_run(c, cfg, R_cap);
  c->stream = (cudaStream_t)cuda_stream;
  RunGeom& g = c->g;
  if (sp.share) {
    g.slot_base = (int32_t)sp.slot_base;
    g.n_init = (int32_t)sp.n_init;
    g.shard = 1;
  }
  int dev = 0;
  if (pa::sweep_supported(g.L) && current_device(&dev) == PA_OK) {
    g.sweep_shape = run_shape(g.L, R_cap, dev);
    int n_sm = 0;
    if (!sp.share && g.model == PA_MODEL_PM1 && !g_sweep_pinned[dev][g.L].load() &&
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      pa::sweep_tail_plan(g.L, g.sweep_shape, cfg->R, n_sm, &g.tail_shape, &g.tail_from);
  }
  for (int p = 0; p < g.n_pop; ++p) {
    make_key(cfg->run_seed, pa::kMetropolis, (uint32_t)p, c->pops[p].key_met);
    make_key(cfg->run_seed, pa::kResample, (uint32_t)p, c->pops[p].key_res);
    make_key(cfg->run_seed, pa::kInit, (uint32_t)p, c->pops[p].key_init);
  }
  const size_t T = (size_t)cfg->n_temps;

  // sizing pass, one stream-ordered allocation, carving pass
  int rc = layout_buffers(c);
  cudaMemPool_t pool = nullptr;
  if (rc == PA_OK) rc = current_device(&dev) == PA_OK ? runs_pool(dev, &pool) : PA_ERR_CUDA;
  if (rc == PA_OK &&
      cudaMallocFromPoolAsync(reinterpret_cast<void**>(&c->slab), c->slab_bytes, pool, c->stream) != cudaSuccess) {
    cudaGetLastError();
    c->slab = nullptr;
    rc = PA_ERR_NOMEM;
  }
  if (rc == PA_OK) rc = layout_buffers(c);
  if (rc != PA_OK) {
    destroy(c);
    return rc;
  }
  cudaStream_t s = c->stream;
  rc = cuda_status(cudaMemsetAsync(c->status, 0, sizeof(int32_t), s));
  if (rc == PA_OK) rc = cuda_status(cudaMemsetAsync(c->qhist, 0, sizeof(unsigned long long) * T * g.q_bins, s));
  for (int p = 0; p < g.n_pop && rc == PA_OK; ++p) {
    rc = cuda_status(cudaMemsetAsync(c->pops[p].hist, 0, sizeof(uint32_t) * T * (size_t)g.n_levels, s));
    if (rc == PA_OK) rc = cuda_status(cudaMemsetAsync(c->pops[p].rec, 0, sizeof(StepRec) * T, s));
    if (rc == PA_OK)  // no stale tile state may carry a step's epoch
      rc = cuda_status(cudaMemsetAsync(c->pops[p].tiles, 0, sizeof(unsigned long long) * (size_t)g.n_count_blocks, s));
    if (rc == PA_OK)
      rc = cuda_status(cudaMemsetAsync(c->pops[p].fhist, 0, sizeof(int32_t) * ((size_t)g.R_cap + 1), s));
    if (rc == PA_OK) rc = cuda_status(cudaMemsetAsync(c->pops[p].fcount, 0, sizeof(int32_t) * 2, s));
    if (rc == PA_OK)  // the block count of the Gaussian model's last-block sums
      rc = cuda_status(cudaMemsetAsync(c->pops[p].ticket, 0, sizeof(int32_t), s));
    if (rc == PA_OK)  // every parent entry is a valid slot at all times, even where a failed step leaves gaps
      rc = cuda_status(cudaMemsetAsync(c->pops[p].parents, 0, sizeof(int32_t) * (size_t)g.pitch, s));
  }
  // Host tables go up in one copy per kind; the +-1 tables' host buffer lives in
  // the run, the Gaussian ones until the stream synchronisation at the end of
  // creation (always taken for that model).
  std::vector<uint32_t> gtab_all;
  std::vector<double> gw_all;
  if (g.model == PA_MODEL_GAUSS) {
    // couplings, and the acceptance and weight tables of every step, on the host
    gauss_couplings(g.L, cfg->disorder_seed, c->Jq_host);
    for (int32_t v : c->Jq_host) c->Jtot += v;
    if (rc == PA_OK) rc = copy_async(c, c->Jq, c->Jq_host.data(), sizeof(int32_t) * c->Jq_host.size());
    if (!c->adaptive && T > 1) {
      const size_t per_tab = (size_t)g.N * pa::kGPatterns;
      gtab_all.assign(T * per_tab, 0u);
      gw_all.assign(T * (size_t)pa::kGTableWeights, 0.0);
      for (size_t t = 1; t < T; ++t) {
        gauss_site_tables(c->Jq_host, g.L, c->betas[t], gtab_all.data() + t * per_tab);
        gauss_weight_tables(c->betas[t] - c->betas[t - 1], gw_all.data() + t * (size_t)pa::kGTableWeights);
      }
      if (rc == PA_OK) rc = copy_async(c, c->gtab, gtab_all.data(), sizeof(uint32_t) * gtab_all.size());
      if (rc == PA_OK) rc = copy_async(c, c->gw, gw_all.data(), sizeof(double) * gw_all.size());
    }
    if (rc == PA_OK) rc = cuda_status(cudaMemsetAsync(c->J, 0, (size_t)3 * g.N, s));
    if (rc == PA_OK) rc = cuda_status(cudaMemsetAsync(c->jtab, 0, sizeof(uint32_t) * 4 * g.N, s));
    if (rc == PA_OK) rc = cuda_status(cudaMemsetAsync(c->qlhist, 0, sizeof(unsigned long long) * T * g.q_bins, s));
    if (rc == PA_OK) rc = launch_rc(pa::launch_init_population(g, c->pops, 0, s));
    if (rc == PA_OK) rc = launch_rc(pa::launch_g_energy_init(g, c->pops, 0, c->Jq, s));
  } else {
    if (!c->adaptive) {
      const std::vector<double> d = distinct_dbetas(c->betas);
      const size_t nl = (size_t)g.n_levels;
      c->wtables_host.resize(d.size() * nl);
      for (size_t i = 0; i < d.size(); ++i) {
        const auto w = cached_weights(g.n_levels, d[i]);
        std::copy(w->begin(), w->end(), c->wtables_host.begin() + (ptrdiff_t)(i * nl));
      }
      if (rc == PA_OK && !d.empty())
        rc = copy_async(c, c->wtables[bits_of(d[0])], c->wtables_host.data(), sizeof(double) * c->wtables_host.size());
    }
    if (rc == PA_OK) rc = launch_rc(pa::launch_init_couplings(g, cfg->disorder_seed, c->J, c->jtab, s));
    if (rc == PA_OK) rc = launch_rc(pa::launch_init_population(g, c->pops, 0, s));
    if (rc == PA_OK) rc = launch_rc(pa::launch_levels_and_hist(g, c->pops, 0, c->jtab, 0, s));
  }
  if (rc == PA_OK) rc = measure(c, 0);
  if (rc == PA_OK) record_step_done(c, 0);
  if (rc == PA_OK && (synchronize || g.model == PA_MODEL_GAUSS)) rc = cuda_status(cudaStreamSynchronize(s));
  if (rc != PA_OK) {
    destroy(c);
    return rc;
  }
  c->t = 0;
  c->done = cfg->n_temps == 1;
  *out = c;
  return PA_OK;
}
}  // namespace

extern "C" {

int pa_create(const pa_config* cfg, void* cuda_stream, pa_ctx** out) try {
  return pa::create_run(cfg, cuda_stream, out, true);
} catch (...) {
  return pa::exception_status();
}

int pa_step(pa_ctx* c) try {
  if (!c) return PA_ERR_INVALID;
  NvtxRange range("pa_step");
  if (c->error != PA_OK) return c->error;
  if (c->done) return PA_DONE;
  const int t = c->t + 1;
  double dbeta;
  if (c->adaptive) {
    int rc = check_device_status(c);
    if (rc == PA_OK) rc = c->model == PA_MODEL_GAUSS ? choose_dbeta_gauss(c, &dbeta) : choose_dbeta(c, &dbeta);
    if (rc != PA_OK) return fail(c, rc);
    double b = c->betas[(size_t)t - 1] + dbeta;
    if (b >= c->cfg.beta_max || dbeta == c->cfg.beta_max - c->betas[(size_t)t - 1]) b = c->cfg.beta_max;
    c->betas[(size_t)t] = b;
  } else {
    dbeta = c->betas[(size_t)t] - c->betas[(size_t)t - 1];
  }
  cudaStream_t s = c->stream;
  int rc = PA_OK;
  for (int p = 0; p < c->g.n_pop && rc == PA_OK; ++p)
    rc = cuda_status(cudaMemsetAsync(c->pops[p].rec + t, 0, sizeof(StepRec), s));
  if (c->model == PA_MODEL_GAUSS) {
    const size_t slot = c->adaptive ? 0 : (size_t)t;
    // the weight tables as the bisection's trials built them, so the resampling's
    // culling fraction is the one the bisection accepted
    if (c->adaptive && rc == PA_OK) rc = launch_rc(pa::launch_g_tables(nullptr, dbeta, c->gw, c->stream));
    if (rc == PA_OK) {
      PhaseTimer pt(c, PA_PHASE_RESAMPLE, 7);
      rc = launch_rc(pa::launch_g_resample(c->g, c->pops, c->cur, t, c->gw + slot * pa::kGTableWeights,
                                           c->status, s));
    }
    // this step's site tables for the beta just chosen, built while the device resamples
    if (c->adaptive && rc == PA_OK) rc = upload_site_tables(c, c->betas[(size_t)t]);
    if (rc == PA_OK) {
      PhaseTimer pt(c, PA_PHASE_SWEEP, 1);
      rc = launch_rc(pa::launch_g_sweep(c->g, c->pops, c->cur, c->jtab, c->Jq, c->Jtot,
                                        c->gtab + slot * c->g.N * pa::kGPatterns, t, c->sweeps[(size_t)t], s));
    }
  } else {
    const double* w = nullptr;
    if (rc == PA_OK) rc = weight_table(c, dbeta, &w);
    uint32_t met[3];
    metropolis_thresholds(c->betas[(size_t)t], met);
    if (rc == PA_OK) {
      PhaseTimer pt(c, PA_PHASE_REWEIGHT, 1);
      rc = launch_rc(pa::launch_reweight(c->g, c->pops, w, t, s));
    }
    if (rc == PA_OK) {
      PhaseTimer pt(c, PA_PHASE_RESAMPLE, 1);
      rc = launch_rc(pa::launch_resample(c->g, c->pops, c->cur, t, c->status, c->lookback, s));
    }
    if (rc == PA_OK && pa::sweep_supported(c->g.L)) {  // per population: the tiles, then a partial last wave's
      PhaseTimer pt(c, PA_PHASE_SWEEP, c->g.n_pop * (c->g.tail_shape >= 0 ? 2 : 1));
      rc = launch_rc(pa::launch_sweep(c->g, c->pops, c->cur, c->jtab, t, c->sweeps[(size_t)t], met, s));
    } else if (rc == PA_OK) {  // lattices beyond a shared-memory tile: sweeps in global memory
      PhaseTimer pt(c, PA_PHASE_SWEEP, c->g.n_pop * (1 + 2 * c->sweeps[(size_t)t]) + 1);
      rc = launch_rc(pa::launch_sweep_global(c->g, c->pops, c->cur, c->jtab, t, c->sweeps[(size_t)t], met, s));
    }
  }
  if (rc != PA_OK) return fail(c, rc);
  c->cur = 1 - c->cur;
  rc = measure(c, t);
  if (rc != PA_OK) return fail(c, rc);
  record_step_done(c, t);
  c->t = t;
  c->stats.steps += 1;
  c->counted_steps.emplace_back(t, c->sweeps[(size_t)t]);
  if (t == c->cfg.n_temps - 1 || (c->adaptive && c->betas[(size_t)t] >= c->cfg.beta_max)) c->done = true;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_debug_lookback(pa_ctx* c, int32_t spins, int32_t withheld_tile) try {
  if (!c || spins < 0 || withheld_tile < -1) return PA_ERR_INVALID;
  c->lookback.spins = spins;
  c->lookback.withheld_tile = withheld_tile;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_debug_bisect(pa_ctx* c, int32_t one_launch, int32_t withheld_block) try {
  if (!c || c->model != PA_MODEL_GAUSS || !c->adaptive || one_launch < 0 || one_launch > 1 || withheld_block < -1 ||
      (!one_launch && withheld_block >= 0))
    return PA_ERR_INVALID;
  c->gbis_blocks = one_launch ? -1 : 0;  // -1: sized again at the next step
  c->gbis_withheld = withheld_block;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_stats_reset(pa_ctx* c, int enable_timing) try {
  if (!c) return PA_ERR_INVALID;
  int rc = cuda_status(cudaStreamSynchronize(c->stream));
  c->stats = pa_stats{};
  c->timing = enable_timing != 0;
  c->timed.clear();
  c->events_used = 0;
  c->counted_steps.clear();
  return rc == PA_OK ? PA_OK : fail(c, rc);
} catch (...) {
  return pa::exception_status();
}

int pa_get_stats(pa_ctx* c, pa_stats* out) try {
  if (!c || !out) return PA_ERR_INVALID;
  int rc = cuda_status(cudaStreamSynchronize(c->stream));
  if (rc != PA_OK) return fail(c, rc);
  pa_stats st = c->stats;
  for (int p = 0; p < PA_N_PHASES; ++p) {
    st.phase_ms[p] = 0.0;
    st.phase_count[p] = 0;
  }
  for (const auto& tm : c->timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, tm.start, tm.end) == cudaSuccess) {
      st.phase_ms[tm.phase] += ms;
      st.phase_count[tm.phase] += 1;
    }
  }
  st.updates = 0;
  for (const auto& ts : c->counted_steps)
    for (int p = 0; p < c->g.n_pop; ++p) {
      int32_t R = 0;
      rc = copy_d2h(c, &R, &c->pops[p].rec[ts.first].R_tilde, sizeof R);
      if (rc != PA_OK) return fail(c, rc);
      st.updates += (int64_t)ts.second * c->g.N * R;
    }
  *out = st;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_sync(pa_ctx* c) try {
  if (!c) return PA_ERR_INVALID;
  int rc = cuda_status(cudaStreamSynchronize(c->stream));
  if (rc == PA_OK) rc = check_device_status(c);
  if (rc != PA_OK) fail(c, rc);
  return c->error;
} catch (...) {
  return pa::exception_status();
}

int pa_run(pa_ctx* c) try {
  if (!c) return PA_ERR_INVALID;
  int rc;
  while ((rc = pa_step(c)) == PA_OK) {
  }
  if (rc != PA_DONE) return rc;
  return pa_sync(c);
} catch (...) {
  return pa::exception_status();
}

int32_t pa_current_step(const pa_ctx* c) { return c ? c->t : -1; }

double pa_beta(const pa_ctx* c, int32_t t) {
  if (!c || t < 0 || t > c->t) return -1.0;
  return c->betas[(size_t)t];
}

int pa_observables(pa_ctx* c, int32_t t, int32_t pop, pa_obs* out) try {
  if (!c || !out || t < 0 || pop < 0 || pop >= c->g.n_pop || c->model != PA_MODEL_PM1) return PA_ERR_INVALID;
  if (t > c->t) return PA_ERR_STATE;
  if (c->error != PA_OK) return c->error;
  // step t's records and histogram, read once step t is done (later steps may run on)
  cudaStream_t st = nullptr;
  int rc = read_stream_for(c, t, &st);
  if (rc != PA_OK) return fail(c, rc);
  const RunGeom& g = c->g;
  std::vector<StepRec> rec((size_t)t + 1);
  std::vector<uint32_t> h((size_t)g.n_levels);
  int32_t flags = 0;
  rc = copy_d2h_on(c, st, rec.data(), c->pops[pop].rec, sizeof(StepRec) * rec.size());
  if (rc == PA_OK)
    rc = copy_d2h_on(c, st, h.data(), c->pops[pop].hist + (size_t)t * g.n_levels, sizeof(uint32_t) * h.size());
  StepRec r0{};
  if (rc == PA_OK && g.n_pop == 2) rc = copy_d2h_on(c, st, &r0, c->pops[0].rec + t, sizeof r0);
  if (rc == PA_OK) rc = copy_d2h_on(c, st, &flags, c->status, sizeof flags);
  if (rc != PA_OK) return fail(c, rc);
  if (flags & pa::kFlagCapacity) return fail(c, PA_ERR_CAPACITY);
  if (flags & pa::kFlagExtinct) return fail(c, PA_ERR_EXTINCT);
  if (flags & pa::kFlagTimeout) return fail(c, PA_ERR_TIMEOUT);
  pm1_observables(g, c->betas, rec.data(), h.data(), t, g.n_pop == 2 ? &r0 : nullptr, out);
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_energy_hist(pa_ctx* c, int32_t t, int32_t pop, int64_t* out, int64_t cap) try {
  if (!c || !out || t < 0 || pop < 0 || pop >= c->g.n_pop || c->model != PA_MODEL_PM1) return PA_ERR_INVALID;
  if (t > c->t) return PA_ERR_STATE;
  if (cap < c->g.n_levels) return PA_ERR_CAPACITY;
  int rc = pa_sync(c);
  if (rc != PA_OK) return rc;
  std::vector<uint32_t> h((size_t)c->g.n_levels);
  rc = copy_d2h(c, h.data(), c->pops[pop].hist + (size_t)t * c->g.n_levels, sizeof(uint32_t) * h.size());
  if (rc != PA_OK) return fail(c, rc);
  for (size_t k = 0; k < h.size(); ++k) out[k] = h[k];
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_q_hist(pa_ctx* c, int32_t t, int64_t* out, int64_t cap) try {
  if (!c || !out || t < 0 || c->g.n_pop != 2) return PA_ERR_INVALID;
  if (t > c->t) return PA_ERR_STATE;
  if (cap < c->g.q_bins) return PA_ERR_CAPACITY;
  int rc = pa_sync(c);
  if (rc != PA_OK) return rc;
  std::vector<unsigned long long> q((size_t)c->g.q_bins);
  rc = copy_d2h(c, q.data(), c->qhist + (size_t)t * c->g.q_bins, sizeof(unsigned long long) * q.size());
  if (rc != PA_OK) return fail(c, rc);
  for (size_t k = 0; k < q.size(); ++k) out[k] = (int64_t)q[k];
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_family_hist(pa_ctx* c, int32_t pop, int64_t cap, int64_t* eta, int64_t* m, int64_t* n) try {
  if (!c || !n || pop < 0 || pop >= c->g.n_pop) return PA_ERR_INVALID;
  int rc = pa_sync(c);
  if (rc != PA_OK) return rc;
  int32_t R = 0;
  rc = copy_d2h(c, &R, &c->pops[pop].rec[c->t].R_tilde, sizeof R);
  if (rc == PA_OK) rc = launch_rc(pa::launch_family_hist(c->g, c->pops, pop, c->cur, c->t, c->stream));
  std::vector<int32_t> mh((size_t)R + 1);
  if (rc == PA_OK)
    rc = copy_d2h(c, mh.data(), c->pops[pop].mhist, sizeof(int32_t) * mh.size());
  if (rc != PA_OK) return fail(c, rc);
  int64_t k = 0;
  for (int64_t e = 1; e <= R; ++e)
    if (mh[(size_t)e] > 0) {
      if (k < cap) {
        if (eta) eta[k] = e;
        if (m) m[k] = mh[(size_t)e];
      }
      ++k;
    }
  *n = k;
  return k <= cap ? PA_OK : PA_ERR_CAPACITY;
} catch (...) {
  return pa::exception_status();
}

int pa_population_size(pa_ctx* c, int32_t pop, int64_t* count) try {
  if (!c || !count || pop < 0 || pop >= c->g.n_pop) return PA_ERR_INVALID;
  int rc = pa_sync(c);
  if (rc != PA_OK) return rc;
  int32_t R = 0;
  rc = copy_d2h(c, &R, &c->pops[pop].rec[c->t].R_tilde, sizeof R);
  if (rc != PA_OK) return fail(c, rc);
  *count = R;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_get_replicas(pa_ctx* c, int32_t pop, int64_t first, int64_t n, int8_t* spins, int32_t* labels,
                    int32_t* energies) try {
  if (!c || pop < 0 || pop >= c->g.n_pop || first < 0 || n < 0) return PA_ERR_INVALID;
  int64_t R = 0;
  int rc = pa_population_size(c, pop, &R);
  if (rc != PA_OK) return rc;
  if (first + n > R) return PA_ERR_INVALID;
  if (n == 0) return PA_OK;
  const RunGeom& g = c->g;
  const PopDev& P = c->pops[pop];
  if (spins) {
    std::vector<int8_t> tmp((size_t)g.N * (size_t)n);
    c->stats.d2h_bytes += (int64_t)g.N * n;
    rc = cuda_status(cudaMemcpy2DAsync(tmp.data(), (size_t)n, P.spins[c->cur] + first, (size_t)g.pitch, (size_t)n,
                                       (size_t)g.N, cudaMemcpyDeviceToHost, c->stream));
    if (rc == PA_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
    if (rc != PA_OK) return fail(c, rc);
    for (int64_t j = 0; j < n; ++j)
      for (int s = 0; s < g.N; ++s) spins[(size_t)j * g.N + s] = tmp[(size_t)s * n + j];
  }
  if (labels) {
    rc = copy_d2h(c, labels, P.labels[c->cur] + first, sizeof(int32_t) * n);
    if (rc != PA_OK) return fail(c, rc);
  }
  if (energies) {
    if (c->model != PA_MODEL_PM1) return PA_ERR_INVALID;
    rc = copy_d2h(c, energies, P.levels + first, sizeof(int32_t) * n);
    if (rc != PA_OK) return fail(c, rc);
    for (int64_t j = 0; j < n; ++j) energies[j] = 2 * energies[j] - 3 * g.N;
  }
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_get_copy_counts(pa_ctx* c, int32_t pop, int32_t* counts, int64_t cap, int64_t* count) try {
  if (!c || !count || pop < 0 || pop >= c->g.n_pop) return PA_ERR_INVALID;
  if (c->t == 0) return PA_ERR_STATE;
  int rc = pa_sync(c);
  if (rc != PA_OK) return rc;
  StepRec r;
  rc = copy_d2h(c, &r, c->pops[pop].rec + c->t, sizeof r);
  if (rc != PA_OK) return fail(c, rc);
  *count = r.R_prev;
  if (r.R_prev > cap) return PA_ERR_CAPACITY;
  if (counts && r.R_prev > 0)
    rc = copy_d2h(c, counts, c->pops[pop].counts, sizeof(int32_t) * r.R_prev);
  return rc == PA_OK ? PA_OK : fail(c, rc);
} catch (...) {
  return pa::exception_status();
}

int pa_get_parents(pa_ctx* c, int32_t pop, int32_t* parents, int64_t cap, int64_t* count) try {
  if (!c || !count || pop < 0 || pop >= c->g.n_pop) return PA_ERR_INVALID;
  if (c->t == 0) return PA_ERR_STATE;
  int64_t R = 0;
  int rc = pa_population_size(c, pop, &R);
  if (rc != PA_OK) return rc;
  *count = R;
  if (R > cap) return PA_ERR_CAPACITY;
  if (parents && R > 0)
    rc = copy_d2h(c, parents, c->pops[pop].parents, sizeof(int32_t) * R);
  return rc == PA_OK ? PA_OK : fail(c, rc);
} catch (...) {
  return pa::exception_status();
}

int pa_get_couplings(pa_ctx* c, int8_t* J, int64_t cap) try {
  if (!c || !J) return PA_ERR_INVALID;
  if (cap < 3 * c->g.N) return PA_ERR_CAPACITY;
  int rc = pa_sync(c);
  if (rc != PA_OK) return rc;
  rc = copy_d2h(c, J, c->J, (size_t)3 * c->g.N);
  return rc == PA_OK ? PA_OK : fail(c, rc);
} catch (...) {
  return pa::exception_status();
}

int pa_destroy(pa_ctx* c) try {
  if (!c) return PA_ERR_INVALID;
  destroy(c);
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_gobservables(pa_ctx* c, int32_t t, int32_t pop, pa_gobs* out) try {
  if (!c || !out || t < 0 || pop < 0 || pop >= c->g.n_pop || c->model != PA_MODEL_GAUSS) return PA_ERR_INVALID;
  if (t > c->t) return PA_ERR_STATE;
  int rc = pa_sync(c);
  if (rc != PA_OK) return rc;
  const RunGeom& g = c->g;
  const int N = g.N;
  std::vector<StepRec> rec((size_t)t + 1);
  std::vector<pa::GRec> gr((size_t)t + 1);
  rc = copy_d2h(c, rec.data(), c->pops[pop].rec, sizeof(StepRec) * rec.size());
  if (rc == PA_OK) rc = copy_d2h(c, gr.data(), c->pops[pop].grec, sizeof(pa::GRec) * gr.size());
  if (rc != PA_OK) return fail(c, rc);
  // Eq. (Q) with weights measured from the lowest energy, Eq. (betaF)
  double lnQ_sum = 0.0, lnQ = 0.0;
  for (int u = 1; u <= t; ++u) {
    const double db = c->betas[(size_t)u] - c->betas[(size_t)u - 1];
    lnQ = std::log(rec[(size_t)u].S_prime / (double)rec[(size_t)u].R_prev) -
          db * ((double)gr[(size_t)u - 1].E_min * 0x1p-20);
    lnQ_sum = lnQ_sum + lnQ;
  }
  const StepRec& r = rec[(size_t)t];
  const pa::GRec& q = gr[(size_t)t];
  pa_gobs o{};
  o.t = t;
  o.beta = c->betas[(size_t)t];
  o.dbeta = t > 0 ? c->betas[(size_t)t] - c->betas[(size_t)t - 1] : 0.0;
  o.R_tilde = r.R_tilde;
  o.sum_E = q.sum_E;
  const unsigned __int128 e2 = ((unsigned __int128)q.sum_E2_hi << 64) | q.sum_E2_lo;
  o.sum_E2 = (double)e2;
  o.E_min = q.E_min;
  o.mean_E = ((double)q.sum_E / (double)o.R_tilde) * 0x1p-20;
  o.var_E = (o.sum_E2 / (double)o.R_tilde) * 0x1p-40 - o.mean_E * o.mean_E;
  o.E_min_prev = t > 0 ? gr[(size_t)t - 1].E_min : 0;
  o.S_prime = t > 0 ? r.S_prime : 0.0;
  o.lnQ = t > 0 ? lnQ : 0.0;
  o.minus_beta_F = (double)N * std::log(2.0) + lnQ_sum;
  o.eps_expected = t > 0 ? r.eps_expected : 0.0;
  o.culled = t > 0 ? r.culled : 0;
  o.sum_eta2 = (int64_t)r.sum_eta2;
  o.n_families = (int64_t)r.n_families;
  o.rho_t = (double)o.sum_eta2 / (double)o.R_tilde;
  o.S_f = -nu_ln_nu(r);
  o.rho_s = (double)o.R_tilde / std::exp(o.S_f);
  o.E0 = q.E0;
  o.g0_tilde = (double)q.n_at_E0 / (double)o.R_tilde;
  o.g0_bar = 2.0 * std::exp(-(o.beta * ((double)q.E0 * 0x1p-20)) - o.minus_beta_F);
  if (g.n_pop == 2) {
    StepRec r0;
    pa::GRec q0;
    rc = copy_d2h(c, &r0, c->pops[0].rec + t, sizeof r0);
    if (rc == PA_OK) rc = copy_d2h(c, &q0, c->pops[0].grec + t, sizeof q0);
    if (rc != PA_OK) return fail(c, rc);
    o.q_pairs = (int64_t)r0.q_pairs;
    o.q_abs_le_02 = (int64_t)r0.q_small;
    o.I02 = o.q_pairs > 0 ? (double)o.q_abs_le_02 / (double)o.q_pairs : 0.0;
    o.ql_sum = q0.ql_sum;
    o.ql_mean = o.q_pairs > 0 ? (double)o.ql_sum / ((double)(3 * (int64_t)N) * (double)o.q_pairs) : 0.0;
    // Eq. (el), and e_l - e of this sample (Eq. KY before the disorder average)
    o.e_l = -(o.beta * 3.0) * (1.0 - o.ql_mean);
    o.delta_KY = o.e_l - o.mean_E / (double)N;
  }
  *out = o;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_get_genergies(pa_ctx* c, int32_t pop, int64_t first, int64_t n, int64_t* E) try {
  if (!c || !E || pop < 0 || pop >= c->g.n_pop || first < 0 || n < 0 || c->model != PA_MODEL_GAUSS)
    return PA_ERR_INVALID;
  int64_t R = 0;
  int rc = pa_population_size(c, pop, &R);
  if (rc != PA_OK) return rc;
  if (first + n > R) return PA_ERR_INVALID;
  if (n == 0) return PA_OK;
  rc = copy_d2h(c, E, c->pops[pop].E64 + first, sizeof(int64_t) * n);
  return rc == PA_OK ? PA_OK : fail(c, rc);
} catch (...) {
  return pa::exception_status();
}

int pa_ql_hist(pa_ctx* c, int32_t t, int64_t* out, int64_t cap) try {
  if (!c || !out || t < 0 || c->model != PA_MODEL_GAUSS || c->g.n_pop != 2) return PA_ERR_INVALID;
  if (t > c->t) return PA_ERR_STATE;
  if (cap < c->g.q_bins) return PA_ERR_CAPACITY;
  int rc = pa_sync(c);
  if (rc != PA_OK) return rc;
  std::vector<unsigned long long> h((size_t)c->g.q_bins);
  rc = copy_d2h(c, h.data(), c->qlhist + (size_t)t * c->g.q_bins, sizeof(unsigned long long) * h.size());
  if (rc != PA_OK) return fail(c, rc);
  for (size_t i = 0; i < h.size(); ++i) out[i] = (int64_t)h[i];
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_get_gcouplings(pa_ctx* c, int32_t* Jq, int64_t cap) try {
  if (!c || !Jq || c->model != PA_MODEL_GAUSS) return PA_ERR_INVALID;
  if (cap < 3 * c->g.N) return PA_ERR_CAPACITY;
  std::memcpy(Jq, c->Jq_host.data(), sizeof(int32_t) * c->Jq_host.size());
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}


int pa_checkpoint(pa_ctx* c, void* buf, size_t cap, size_t* size) try {
  if (!c || !size) return PA_ERR_INVALID;
  int rc = pa_sync(c);
  if (rc != PA_OK) return rc;
  const RunGeom& g = c->g;
  const int t = c->t;
  int32_t Rt[2] = {0, 0}, Rp[2] = {0, 0};
  for (int p = 0; p < g.n_pop; ++p) {
    StepRec r;
    rc = copy_d2h(c, &r, c->pops[p].rec + t, sizeof r);
    if (rc != PA_OK) return fail(c, rc);
    Rt[p] = r.R_tilde;
    Rp[p] = t > 0 ? r.R_prev : 0;
  }
  const bool gauss = c->model == PA_MODEL_GAUSS;
  const size_t need = ckpt_bytes(g, c->model, t, c->cfg.n_temps, Rt, Rp);
  *size = need;
  if (!buf || cap < need) return PA_ERR_CAPACITY;
  char* o = static_cast<char*>(buf);
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, sizeof h.magic);
  h.version = kCkptVersion;
  h.header_bytes = sizeof(CkptHeader);
  h.L = g.L;
  h.n_pop = g.n_pop;
  h.q_bins = g.q_bins;
  h.n_temps = c->cfg.n_temps;
  h.R = c->cfg.R;
  h.R_cap = c->cfg.R_cap;
  h.disorder_seed = c->cfg.disorder_seed;
  h.run_seed = c->cfg.run_seed;
  h.eps_target = c->adaptive ? c->cfg.eps_target : 0.0;
  h.beta_max = c->adaptive ? c->cfg.beta_max : 0.0;
  h.t = t;
  h.done = c->done ? 1 : 0;
  h.adaptive = c->adaptive ? 1 : 0;
  h.n_sweeps = c->cfg.n_sweeps;
  for (int p = 0; p < 2; ++p) {
    h.R_tilde[p] = Rt[p];
    h.R_prev[p] = Rp[p];
  }
  h.model = c->model;
  h.total_bytes = need;
  std::memcpy(o, &h, sizeof h);
  o += sizeof h;
  std::memcpy(o, c->betas.data(), sizeof(double) * (size_t)c->cfg.n_temps);
  o += sizeof(double) * (size_t)c->cfg.n_temps;
  std::memcpy(o, c->sweeps.data(), sizeof(int32_t) * (size_t)c->cfg.n_temps);
  o += sizeof(int32_t) * (size_t)c->cfg.n_temps;
  for (int p = 0; p < g.n_pop && rc == PA_OK; ++p) {
    const PopDev& P = c->pops[p];
    const size_t R = (size_t)Rt[p];
    auto get = [&](const void* src, size_t bytes) {
      if (rc == PA_OK && bytes) rc = copy_d2h(c, o, src, bytes);
      o += bytes;
    };
    get(P.rec, sizeof(StepRec) * (size_t)(t + 1));
    if (gauss)
      get(P.grec, sizeof(pa::GRec) * (size_t)(t + 1));
    else
      get(P.hist, sizeof(uint32_t) * (size_t)(t + 1) * (size_t)g.n_levels);
    if (rc == PA_OK && R) {
      c->stats.d2h_bytes += (int64_t)(g.N * R);
      rc = cuda_status(cudaMemcpy2DAsync(o, R, P.spins[c->cur], (size_t)g.pitch, R, (size_t)g.N,
                                         cudaMemcpyDeviceToHost, c->stream));
      if (rc == PA_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
    }
    o += (size_t)g.N * R;
    get(P.labels[c->cur], sizeof(int32_t) * R);
    if (gauss)
      get(P.E64, sizeof(int64_t) * R);
    else
      get(P.levels, sizeof(int32_t) * R);
    get(P.counts, sizeof(int32_t) * (size_t)Rp[p]);
    get(P.parents, sizeof(int32_t) * R);
    if (rc == PA_OK) rc = launch_rc(pa::launch_family_hist(g, c->pops, p, c->cur, t, c->stream));
    get(P.mhist, sizeof(int32_t) * (R + 1));
  }
  const size_t qbytes = sizeof(unsigned long long) * (size_t)(t + 1) * (size_t)g.q_bins;
  if (rc == PA_OK) rc = copy_d2h(c, o, c->qhist, qbytes);
  if (rc == PA_OK && gauss) rc = copy_d2h(c, o + qbytes, c->qlhist, qbytes);
  return rc == PA_OK ? PA_OK : fail(c, rc);
} catch (...) {
  return pa::exception_status();
}

int pa_restore(const pa_config* cfg, const void* buf, size_t size, void* cuda_stream, pa_ctx** out) try {
  if (!out) return PA_ERR_INVALID;
  *out = nullptr;
  if (!cfg || !buf || size < sizeof(CkptHeader)) return PA_ERR_INVALID;
  CkptHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, kCkptMagic, sizeof h.magic) != 0 || h.version != kCkptVersion ||
      h.header_bytes != sizeof(CkptHeader) || h.total_bytes != size)
    return PA_ERR_INVALID;
  const int64_t R_cap = capacity_of(cfg);
  const bool adaptive = cfg->betas == nullptr;
  if (h.model != cfg->model) return PA_ERR_INVALID;
  const bool gauss = cfg->model == PA_MODEL_GAUSS;
  if (h.L != cfg->L || h.n_pop != cfg->n_pop || h.q_bins != cfg->q_bins || h.n_temps != cfg->n_temps ||
      h.R != cfg->R || h.R_cap != R_cap || h.disorder_seed != cfg->disorder_seed || h.run_seed != cfg->run_seed ||
      h.adaptive != (adaptive ? 1 : 0) || h.n_sweeps != cfg->n_sweeps || h.t < 0 || h.t >= h.n_temps ||
      (adaptive && (h.eps_target != cfg->eps_target || h.beta_max != cfg->beta_max)))
    return PA_ERR_INVALID;
  pa_ctx* c = nullptr;
  int rc = pa_create(cfg, cuda_stream, &c);
  if (rc != PA_OK) return rc;
  const RunGeom& g = c->g;
  const int t = h.t;
  for (int p = 0; p < g.n_pop; ++p)
    if (h.R_tilde[p] < 1 || h.R_tilde[p] > g.R_cap || h.R_prev[p] < 0 || h.R_prev[p] > g.R_cap) {
      pa_destroy(c);
      return PA_ERR_INVALID;
    }
  if (ckpt_bytes(g, h.model, t, h.n_temps, h.R_tilde, h.R_prev) != size) {
    pa_destroy(c);
    return PA_ERR_INVALID;
  }
  const char* in = static_cast<const char*>(buf) + sizeof h;
  const double* betas = reinterpret_cast<const double*>(in);
  in += sizeof(double) * (size_t)h.n_temps;
  const int32_t* sweeps = reinterpret_cast<const int32_t*>(in);
  in += sizeof(int32_t) * (size_t)h.n_temps;
  // the schedule must be the one the checkpoint was taken with
  for (int u = 0; u < h.n_temps; ++u) {
    if (!adaptive && std::memcmp(&betas[u], &c->betas[(size_t)u], sizeof(double)) != 0) rc = PA_ERR_INVALID;
    if (sweeps[u] != c->sweeps[(size_t)u]) rc = PA_ERR_INVALID;
  }
  if (rc != PA_OK) {
    pa_destroy(c);
    return rc;
  }
  if (!ckpt_payload_ok(g, gauss, t, h.R, h, in)) {
    pa_destroy(c);
    return PA_ERR_INVALID;
  }
  for (int u = 0; u <= t; ++u) c->betas[(size_t)u] = betas[u];
  c->cur = 0;
  for (int p = 0; p < g.n_pop && rc == PA_OK; ++p) {
    PopDev& P = c->pops[p];
    const size_t R = (size_t)h.R_tilde[p];
    auto put = [&](void* dst, size_t bytes) {
      if (rc == PA_OK && bytes) rc = copy_h2d(c, dst, in, bytes);
      in += bytes;
    };
    put(P.rec, sizeof(StepRec) * (size_t)(t + 1));
    if (gauss)
      put(P.grec, sizeof(pa::GRec) * (size_t)(t + 1));
    else
      put(P.hist, sizeof(uint32_t) * (size_t)(t + 1) * (size_t)g.n_levels);
    if (rc == PA_OK) {
      c->stats.h2d_bytes += (int64_t)(g.N * R);
      rc = cuda_status(cudaMemcpy2DAsync(P.spins[0], (size_t)g.pitch, in, R, R, (size_t)g.N,
                                         cudaMemcpyHostToDevice, c->stream));
      if (rc == PA_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
    }
    in += (size_t)g.N * R;
    put(P.labels[0], sizeof(int32_t) * R);
    if (gauss)
      put(P.E64, sizeof(int64_t) * R);
    else
      put(P.levels, sizeof(int32_t) * R);
    put(P.counts, sizeof(int32_t) * (size_t)h.R_prev[p]);
    put(P.parents, sizeof(int32_t) * R);
    put(P.mhist, sizeof(int32_t) * (R + 1));
  }
  const size_t qbytes = sizeof(unsigned long long) * (size_t)(t + 1) * (size_t)g.q_bins;
  if (rc == PA_OK) rc = copy_h2d(c, c->qhist, in, qbytes);
  if (rc == PA_OK && gauss) rc = copy_h2d(c, c->qlhist, in + qbytes, qbytes);
  if (rc != PA_OK) {
    pa_destroy(c);
    return rc;
  }
  c->t = t;
  c->done = h.done != 0;
  *out = c;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_sweep_shapes(int32_t L, pa_sweep_shape* shapes, int32_t cap, int32_t* n) try {
  if (!n || cap < 0 || (cap > 0 && !shapes) || !pa::sweep_supported(L)) return PA_ERR_INVALID;
  const int k = pa::sweep_shape_count(L);
  *n = k;
  for (int i = 0; i < k && i < cap; ++i) {
    pa::SweepShapeInfo si{};
    pa::sweep_shape_info(L, i, &si);
    shapes[i].L = si.L;
    shapes[i].words = si.W;
    shapes[i].threads = si.NT;
    shapes[i].ctas_per_sm = si.MB;
    shapes[i].smem_bytes = si.smem;
  }
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_sweep_select(int32_t L, int32_t index) try {
  if (!pa::sweep_supported(L) || index < -1 || index >= pa::sweep_shape_count(L)) return PA_ERR_INVALID;
  int dev = 0;
  const int rc = current_device(&dev);
  if (rc != PA_OK) return rc;
  g_sweep_choice[dev][L].store(index < 0 ? 0 : index);
  g_sweep_pinned[dev][L].store(index >= 0);
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_sweep_selected(int32_t L, int32_t* index) try {
  if (!index || !pa::sweep_supported(L)) return PA_ERR_INVALID;
  int dev = 0;
  const int rc = current_device(&dev);
  if (rc != PA_OK) return rc;
  *index = g_sweep_choice[dev][L].load();
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_sweep_plan(const pa_ctx* c, int32_t* shape, int32_t* tail_shape, int32_t* tail_from) try {
  if (!c || !shape || !tail_shape || !tail_from) return PA_ERR_INVALID;
  *shape = c->g.sweep_shape;
  *tail_shape = c->g.tail_shape;
  *tail_from = c->g.tail_from;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_sweep_autotune(int32_t L, int32_t R, int32_t launches, double* ms_per_launch, int32_t cap, int32_t* best) try {
  if (!best || !pa::sweep_supported(L) || R < 1 || launches < 1 || cap < 0 || (cap > 0 && !ms_per_launch))
    return PA_ERR_INVALID;
  int dev = 0;
  int rc = current_device(&dev);
  if (rc != PA_OK) return rc;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return PA_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rc = cuda_status(cudaEventCreate(&e0));
  if (rc == PA_OK) rc = cuda_status(cudaEventCreate(&e1));
  // scratch run: one step from beta 0 to 0.5 leaves a resampled population whose
  // sweep can be relaunched (it reads one buffer and rewrites the other)
  const double betas[2] = {0.0, 0.5};
  pa_config cfg{};
  cfg.L = L;
  cfg.n_pop = 1;
  cfg.R = R;
  cfg.disorder_seed = 1;
  cfg.run_seed = 1;
  cfg.n_temps = 2;
  cfg.betas = betas;
  cfg.n_sweeps = 10;
  cfg.q_bins = 65;
  pa_ctx* c = nullptr;
  if (rc == PA_OK) rc = pa_create(&cfg, s, &c);
  if (rc == PA_OK) rc = pa_step(c);
  if (rc == PA_OK) rc = pa_sync(c);
  int best_i = -1;
  double best_ms = 0.0;
  if (rc == PA_OK) {
    uint32_t met[3];
    metropolis_thresholds(betas[1], met);
    const int src = 1 - c->cur;  // the buffer the step's sweep gathered from
    const int n = pa::sweep_shape_count(L);
    for (int i = 0; i < n && rc == PA_OK; ++i) {
      c->g.sweep_shape = i;
      c->g.tail_shape = -1;
      double t_ms = -1.0;
      int e = pa::launch_sweep(c->g, c->pops, src, c->jtab, 1, cfg.n_sweeps, met, s);
      if (e == 0) {
        cudaEventRecord(e0, s);
        for (int k = 0; k < launches && e == 0; ++k) e = pa::launch_sweep(c->g, c->pops, src, c->jtab, 1, cfg.n_sweeps, met, s);
        cudaEventRecord(e1, s);
        rc = cuda_status(cudaEventSynchronize(e1));
        float f = 0.f;
        if (rc == PA_OK && e == 0 && cudaEventElapsedTime(&f, e0, e1) == cudaSuccess) t_ms = (double)f / launches;
      }
      if (e != 0) cudaGetLastError();  // a shape that does not fit this device: skipped
      if (ms_per_launch && i < cap) ms_per_launch[i] = t_ms;
      if (t_ms >= 0.0 && (best_i < 0 || t_ms < best_ms)) {
        best_i = i;
        best_ms = t_ms;
      }
    }
  }
  if (c) pa_destroy(c);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (rc != PA_OK) return rc;
  if (best_i < 0) return PA_ERR_CUDA;
  g_sweep_choice[dev][L].store(best_i);
  g_sweep_pinned[dev][L].store(false);
  *best = best_i;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

}  // extern "C"

// ---------------------------------------------------------------- sharded runs
//
// One rank's share of a population split across ranks (pa.h, pa_shard_*): the
// rank's slots live in an ordinary run (pa_ctx) whose global slot base makes every
// random word the one-process run's; the exchanges between the phases of a step go
// through the caller's host functions (pa_comm).

struct pa_shard {
  pa_ctx* c = nullptr;
  pa_comm comm{};
  int32_t rank = 0, n_ranks = 1;
  int64_t lo = 0, hi = 0;                          // this rank's global slots [lo, hi)
  int64_t R_glob[2] = {0, 0};                      // global population sizes of the current step
  std::vector<StepRec> rec[2];                     // global step records of steps 0..t
  std::vector<uint32_t> hist[2];                   // global level histograms, (t + 1) x n_levels
  std::vector<std::vector<int64_t>> qhist;         // global overlap histograms
  long long* dscratch = nullptr;                   // device: family edges (8), entropy sum (2)
  int32_t* dsizes = nullptr;                       // device: family sizes and their counts
};

namespace {

// Rank q's global slots [lo, hi) of a population cut from R slots: whole units of
// 1024 slots (tiles and Philox word groups stay aligned with the global ones).
void shard_block(int64_t R, int P, int q, int64_t* lo, int64_t* hi) {
  const int64_t units = (R + 1023) / 1024;
  *lo = std::min<int64_t>(R, 1024 * ((units * q) / P));
  *hi = std::min<int64_t>(R, 1024 * ((units * (q + 1)) / P));
}

int comm_rc(int e) { return e == 0 ? PA_OK : PA_ERR_CUDA; }

// The device status of one rank's run after its resampling: a rank may hold no
// old slots, or receive no copies, while the population lives on other ranks, so
// the extinction flag is cleared here (the step checks the global size instead).
int shard_status(pa_ctx* c) {
  int32_t flags = 0;
  int rc = cuda_status(cudaStreamSynchronize(c->stream));
  if (rc == PA_OK) rc = copy_d2h(c, &flags, c->status, sizeof flags);
  if (rc == PA_OK && (flags & pa::kFlagExtinct)) {
    const int32_t kept = flags & ~pa::kFlagExtinct;
    rc = copy_h2d(c, c->status, &kept, sizeof kept);
  }
  if (rc != PA_OK) return rc;
  if (flags & pa::kFlagCapacity) return PA_ERR_CAPACITY;
  if (flags & pa::kFlagTimeout) return PA_ERR_TIMEOUT;
  return PA_OK;
}

// Families of population p at step t over all ranks, and the global family
// statistics in r: local runs, the ranks' first and last runs joined in rank order
// (a family may span ranks), the global size histogram, and the entropy sum by the
// device code of the one-process run.
int shard_families(pa_shard* s, int p, int t, StepRec& r) {
  pa_ctx* c = s->c;
  const RunGeom& g = c->g;
  const int P = s->n_ranks;
  int rc = launch_rc(pa::launch_shard_families(g, c->pops, p, c->cur, t, s->dscratch, c->stream));
  long long edge[8];
  std::vector<int32_t> mh((size_t)g.R_cap + 1);
  if (rc == PA_OK) rc = copy_d2h(c, edge, s->dscratch, sizeof edge);
  if (rc == PA_OK) rc = copy_d2h(c, mh.data(), c->pops[p].mhist, sizeof(int32_t) * mh.size());
  if (rc != PA_OK) return rc;
  std::vector<int64_t> mine(edge, edge + 8), all((size_t)P * 8);
  rc = comm_rc(s->comm.allgather_i64(s->comm.user, mine.data(), 8, all.data()));
  std::vector<int64_t> m(mh.begin(), mh.end());
  if (rc == PA_OK) rc = comm_rc(s->comm.allreduce_i64(s->comm.user, m.data(), (int64_t)m.size()));
  if (rc != PA_OK) return rc;
  // join the edge runs in rank order
  std::vector<int64_t> joined;
  bool open = false;
  int64_t open_lab = 0, open_len = 0, s2 = 0, nf = 0;
  for (int q = 0; q < P; ++q) {
    const int64_t* e = &all[(size_t)q * 8];
    s2 += e[6];
    nf += e[7];
    if (!e[0]) continue;
    const int64_t f = e[1], lf = e[2], l = e[3], ll = e[4], runs = e[5];
    if (runs == 1) {  // the rank's slots are one run
      if (open && f == open_lab) {
        open_len += lf;
      } else {
        if (open) joined.push_back(open_len);
        open = true;
        open_lab = f;
        open_len = lf;
      }
      continue;
    }
    if (open && f == open_lab) {
      joined.push_back(open_len + lf);
    } else {
      if (open) joined.push_back(open_len);
      joined.push_back(lf);
    }
    open = true;
    open_lab = l;
    open_len = ll;
  }
  if (open) joined.push_back(open_len);
  for (int64_t eta : joined) {
    if (eta < 1 || eta >= (int64_t)m.size()) return PA_ERR_INVALID;
    m[(size_t)eta] += 1;
    s2 += eta * eta;
    nf += 1;
  }
  std::vector<int32_t> eta_k, m_k;
  for (size_t e = 1; e < m.size(); ++e)
    if (m[e] > 0) {
      eta_k.push_back((int32_t)e);
      m_k.push_back((int32_t)m[e]);
    }
  const int K = (int)eta_k.size();
  if (K > 0) {
    rc = copy_h2d(c, s->dsizes, eta_k.data(), sizeof(int32_t) * (size_t)K);
    if (rc == PA_OK) rc = copy_h2d(c, s->dsizes + g.R_cap + 1, m_k.data(), sizeof(int32_t) * (size_t)K);
    if (rc == PA_OK)
      rc = launch_rc(pa::launch_entropy_of_sizes(s->dsizes, s->dsizes + g.R_cap + 1, K, (int)r.R_tilde,
                                                 s->dscratch + 8, c->stream));
    long long nll[2] = {0, 0};
    if (rc == PA_OK) rc = copy_d2h(c, nll, s->dscratch + 8, sizeof nll);
    if (rc != PA_OK) return rc;
    r.nll_hi = nll[0];
    r.nll_lo = (unsigned long long)nll[1];
  }
  r.sum_eta2 = (unsigned long long)s2;
  r.n_families = (unsigned long long)nf;
  return PA_OK;
}

// The measurements of step t over all ranks: level histograms, families, overlap.
int shard_measure(pa_shard* s, int t) {
  pa_ctx* c = s->c;
  const RunGeom& g = c->g;
  int rc = PA_OK;
  for (int p = 0; p < g.n_pop && rc == PA_OK; ++p) {
    std::vector<uint32_t> h((size_t)g.n_levels);
    uint32_t* dh = c->pops[p].hist + (size_t)t * g.n_levels;
    rc = copy_d2h(c, h.data(), dh, sizeof(uint32_t) * h.size());
    std::vector<int64_t> v(h.begin(), h.end());
    if (rc == PA_OK) rc = comm_rc(s->comm.allreduce_i64(s->comm.user, v.data(), (int64_t)v.size()));
    if (rc != PA_OK) break;
    for (size_t k = 0; k < h.size(); ++k) h[k] = (uint32_t)v[k];
    rc = copy_h2d(c, dh, h.data(), sizeof(uint32_t) * h.size());  // the next step's tables need the global one
    s->hist[p].insert(s->hist[p].end(), h.begin(), h.end());
    StepRec& r = s->rec[p][(size_t)t];
    r.R_tilde = (int32_t)s->R_glob[p];
    if (rc == PA_OK) rc = shard_families(s, p, t, r);
  }
  if (rc == PA_OK && g.n_pop == 2) {
    // the overlap kernel adds to its outputs (a share's creation has measured step 0 once already)
    rc = cuda_status(cudaMemsetAsync(c->qhist + (size_t)t * g.q_bins, 0, sizeof(unsigned long long) * g.q_bins,
                                     c->stream));
    if (rc == PA_OK)
      rc = cuda_status(cudaMemsetAsync(&c->pops[0].rec[t].q_small, 0, sizeof(unsigned long long), c->stream));
    if (rc == PA_OK) rc = launch_rc(pa::launch_overlap(g, c->pops, c->cur, t, c->qhist, c->stream));
    std::vector<unsigned long long> q((size_t)g.q_bins);
    StepRec r0{};
    if (rc == PA_OK) rc = copy_d2h(c, q.data(), c->qhist + (size_t)t * g.q_bins, sizeof(unsigned long long) * q.size());
    if (rc == PA_OK) rc = copy_d2h(c, &r0, c->pops[0].rec + t, sizeof r0);
    std::vector<int64_t> v(q.begin(), q.end());
    v.push_back((int64_t)r0.q_small);
    if (rc == PA_OK) rc = comm_rc(s->comm.allreduce_i64(s->comm.user, v.data(), (int64_t)v.size()));
    if (rc == PA_OK) {
      s->rec[0][(size_t)t].q_small = (unsigned long long)v.back();
      s->rec[0][(size_t)t].q_pairs = (unsigned long long)std::min(s->R_glob[0], s->R_glob[1]);
      v.pop_back();
      s->qhist.push_back(v);
    }
  }
  return rc;
}

// Moves every copy of population p to the rank that holds its new slot: rank r's
// copies are the global new slots [off[r], off[r] + tot[r]), already written out in
// order at local slots [0, tot[r]) of the other buffer; rank q receives those in
// [LO_q, HI_q).  Pairs of ranks exchange in rank order (the lower rank sends
// first), each message a count, the copies' spins (N rows) and their labels.  The
// new local population goes to the current buffer (spins) and the other (labels).
int shard_exchange(pa_shard* s, int p, const std::vector<int64_t>& off, const std::vector<int64_t>& tot,
                   int64_t R_new, int64_t R_part, int64_t* n_local) {
  pa_ctx* c = s->c;
  const RunGeom& g = c->g;
  const PopDev& P = c->pops[p];
  const int r = s->rank, Pn = s->n_ranks;
  int64_t LO, HI;
  shard_block(R_part, Pn, r, &LO, &HI);
  HI = std::min(HI, R_new);
  const int64_t n_new = std::max<int64_t>(0, HI - std::max<int64_t>(LO, 0));
  const int64_t N = g.N;
  std::vector<int8_t> rs((size_t)(N * std::max<int64_t>(n_new, 1)));
  std::vector<int32_t> rl((size_t)std::max<int64_t>(n_new, 1));
  auto range_to = [&](int q, int64_t* a, int64_t* b) {  // my local copies that rank q holds
    int64_t lq, hq;
    shard_block(R_part, Pn, q, &lq, &hq);
    hq = std::min(hq, R_new);
    const int64_t ga = std::max(off[(size_t)r], lq), gb = std::min(off[(size_t)r] + tot[(size_t)r], hq);
    *a = ga - off[(size_t)r];
    *b = std::max(*a, gb - off[(size_t)r]);
  };
  auto pack = [&](int64_t a, int64_t b, std::vector<int8_t>& sp, std::vector<int32_t>& lb) {
    const int64_t n = b - a;
    sp.assign((size_t)(N * std::max<int64_t>(n, 1)), 0);
    lb.assign((size_t)std::max<int64_t>(n, 1), 0);
    if (n == 0) return PA_OK;
    int rc = cuda_status(cudaMemcpy2DAsync(sp.data(), (size_t)n, P.spins[1 - c->cur] + a, (size_t)g.pitch, (size_t)n,
                                           (size_t)N, cudaMemcpyDeviceToHost, c->stream));
    if (rc == PA_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
    if (rc == PA_OK) rc = copy_d2h(c, lb.data(), P.labels[1 - c->cur] + a, sizeof(int32_t) * (size_t)n);
    return rc;
  };
  auto place = [&](int q, int64_t n, const int8_t* sp, const int32_t* lb) {  // copies from rank q
    const int64_t at = std::max(off[(size_t)q], LO) - LO;
    if (n == 0) return PA_OK;
    if (at < 0 || at + n > n_new) return PA_ERR_INVALID;
    for (int64_t site = 0; site < N; ++site)
      std::memcpy(&rs[(size_t)(site * n_new + at)], sp + site * n, (size_t)n);
    std::memcpy(&rl[(size_t)at], lb, sizeof(int32_t) * (size_t)n);
    return PA_OK;
  };
  int rc = PA_OK;
  std::vector<int8_t> sp;
  std::vector<int32_t> lb;
  for (int q = 0; q < Pn && rc == PA_OK; ++q) {
    int64_t a, b;
    range_to(q, &a, &b);
    if (q == r) {
      rc = pack(a, b, sp, lb);
      if (rc == PA_OK) rc = place(q, b - a, sp.data(), lb.data());
      continue;
    }
    auto send_to = [&]() {
      int e = pack(a, b, sp, lb);
      const int64_t n = b - a;
      if (e == PA_OK) e = comm_rc(s->comm.send(s->comm.user, q, &n, sizeof n));
      if (e == PA_OK && n > 0) e = comm_rc(s->comm.send(s->comm.user, q, sp.data(), N * n));
      if (e == PA_OK && n > 0) e = comm_rc(s->comm.send(s->comm.user, q, lb.data(), (int64_t)sizeof(int32_t) * n));
      return e;
    };
    auto recv_from = [&]() {
      int64_t n = 0;
      int e = comm_rc(s->comm.recv(s->comm.user, q, &n, sizeof n));
      if (e != PA_OK) return e;
      if (n < 0 || n > n_new) return PA_ERR_INVALID;
      std::vector<int8_t> rsp((size_t)(N * std::max<int64_t>(n, 1)));
      std::vector<int32_t> rlb((size_t)std::max<int64_t>(n, 1));
      if (n > 0) e = comm_rc(s->comm.recv(s->comm.user, q, rsp.data(), N * n));
      if (e == PA_OK && n > 0) e = comm_rc(s->comm.recv(s->comm.user, q, rlb.data(), (int64_t)sizeof(int32_t) * n));
      if (e == PA_OK) e = place(q, n, rsp.data(), rlb.data());
      return e;
    };
    if (r < q) {
      rc = send_to();
      if (rc == PA_OK) rc = recv_from();
    } else {
      rc = recv_from();
      if (rc == PA_OK) rc = send_to();
    }
  }
  if (rc != PA_OK) return rc;
  if (n_new > 0) {
    rc = cuda_status(cudaMemcpy2DAsync(P.spins[c->cur], (size_t)g.pitch, rs.data(), (size_t)n_new, (size_t)n_new,
                                       (size_t)N, cudaMemcpyHostToDevice, c->stream));
    if (rc == PA_OK) rc = copy_h2d(c, P.labels[1 - c->cur], rl.data(), sizeof(int32_t) * (size_t)n_new);
    std::vector<int32_t> iota((size_t)n_new);
    for (int64_t j = 0; j < n_new; ++j) iota[(size_t)j] = (int32_t)j;
    if (rc == PA_OK) rc = copy_h2d(c, P.parents, iota.data(), sizeof(int32_t) * (size_t)n_new);
  }
  *n_local = n_new;
  return rc;
}

}  // namespace

extern "C" {

int pa_shard_create(const pa_config* cfg, int32_t rank, int32_t n_ranks, const pa_comm* comm, void* cuda_stream,
                    pa_shard** out) try {
  if (!out) return PA_ERR_INVALID;
  *out = nullptr;
  if (!cfg || !comm || !comm->allreduce_i64 || !comm->allgather_i64 || !comm->send || !comm->recv || n_ranks < 1 ||
      rank < 0 || rank >= n_ranks || cfg->model != PA_MODEL_PM1 || !cfg->betas || !pa::sweep_supported(cfg->L))
    return PA_ERR_INVALID;
  pa_shard* s = new (std::nothrow) pa_shard();
  if (!s) return PA_ERR_NOMEM;
  s->comm = *comm;
  s->rank = rank;
  s->n_ranks = n_ranks;
  shard_block(cfg->R, n_ranks, rank, &s->lo, &s->hi);
  int rc = pa::create_run_share(cfg, cuda_stream, &s->c, s->lo, s->hi - s->lo);
  const RunGeom* g = s->c ? &s->c->g : nullptr;
  if (rc == PA_OK && (cudaMalloc(reinterpret_cast<void**>(&s->dscratch), sizeof(long long) * 10) != cudaSuccess ||
                      cudaMalloc(reinterpret_cast<void**>(&s->dsizes), sizeof(int32_t) * 2 * ((size_t)g->R_cap + 1)) !=
                          cudaSuccess)) {
    cudaGetLastError();
    rc = PA_ERR_NOMEM;
  }
  if (rc == PA_OK) {
    for (int p = 0; p < cfg->n_pop; ++p) {
      s->R_glob[p] = cfg->R;
      s->rec[p].assign((size_t)cfg->n_temps, StepRec{});
    }
    rc = shard_measure(s, 0);
  }
  if (rc != PA_OK) {
    pa_shard_destroy(s);
    return rc;
  }
  *out = s;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_shard_step(pa_shard* s) try {
  if (!s) return PA_ERR_INVALID;
  pa_ctx* c = s->c;
  if (c->error != PA_OK) return c->error;
  if (c->done) return PA_DONE;
  RunGeom& g = c->g;
  const int t = c->t + 1, np = g.n_pop, Pn = s->n_ranks;
  const double dbeta = c->betas[(size_t)t] - c->betas[(size_t)t - 1];
  cudaStream_t st = c->stream;
  int rc = PA_OK;
  for (int p = 0; p < np && rc == PA_OK; ++p) rc = cuda_status(cudaMemsetAsync(c->pops[p].rec + t, 0, sizeof(StepRec), st));
  // 1-2. tables from the global histogram of step t-1; copy numbers of the local old
  // slots (their uniforms addressed by global slot) and the copies in local order
  const double* w = nullptr;
  if (rc == PA_OK) rc = weight_table(c, dbeta, &w);
  g.slot_base = (int32_t)s->lo;
  if (rc == PA_OK) rc = launch_rc(pa::launch_reweight(g, c->pops, w, t, st));
  if (rc == PA_OK) rc = launch_rc(pa::launch_resample(g, c->pops, c->cur, t, c->status, c->lookback, st));
  for (int p = 0; p < np && rc == PA_OK; ++p) rc = launch_rc(pa::launch_copy_parents(g, c->pops, p, c->cur, t, st));
  if (rc == PA_OK) rc = shard_status(c);
  StepRec loc[2];
  for (int p = 0; p < np && rc == PA_OK; ++p) rc = copy_d2h(c, &loc[p], c->pops[p].rec + t, sizeof(StepRec));
  if (rc != PA_OK) return fail(c, rc);
  // 3. global offsets: the ranks' copy totals in rank order
  std::vector<int64_t> mine((size_t)2 * np), all((size_t)2 * np * Pn);
  for (int p = 0; p < np; ++p) {
    mine[(size_t)2 * p] = loc[p].R_tilde;
    mine[(size_t)2 * p + 1] = loc[p].culled;
  }
  rc = comm_rc(s->comm.allgather_i64(s->comm.user, mine.data(), 2 * np, all.data()));
  if (rc != PA_OK) return fail(c, rc);
  std::vector<int64_t> off[2], tot[2];
  int64_t R_new[2] = {0, 0}, culled[2] = {0, 0}, R_part = 0;
  for (int p = 0; p < np; ++p) {
    for (int q = 0; q < Pn; ++q) {
      off[p].push_back(R_new[p]);
      tot[p].push_back(all[(size_t)(q * 2 * np + 2 * p)]);
      R_new[p] += tot[p].back();
      culled[p] += all[(size_t)(q * 2 * np + 2 * p + 1)];
    }
    if (R_new[p] > g.R_cap) return fail(c, PA_ERR_CAPACITY);
    if (R_new[p] == 0) return fail(c, PA_ERR_EXTINCT);
    R_part = std::max(R_part, R_new[p]);
  }
  // 4. every copy to the rank that holds its new slot
  int64_t n_local[2] = {0, 0};
  for (int p = 0; p < np && rc == PA_OK; ++p) rc = shard_exchange(s, p, off[p], tot[p], R_new[p], R_part, &n_local[p]);
  for (int p = 0; p < np && rc == PA_OK; ++p) {
    const int32_t n = (int32_t)n_local[p];
    rc = copy_h2d(c, &c->pops[p].rec[t].R_tilde, &n, sizeof n);
  }
  if (rc != PA_OK) return fail(c, rc);
  int64_t hi;
  shard_block(R_part, Pn, s->rank, &s->lo, &hi);
  // 5. sweeps of the local slots (Metropolis words addressed by global slot)
  g.slot_base = (int32_t)s->lo;
  uint32_t met[3];
  metropolis_thresholds(c->betas[(size_t)t], met);
  rc = launch_rc(pa::launch_sweep(g, c->pops, c->cur, c->jtab, t, c->sweeps[(size_t)t], met, st));
  if (rc != PA_OK) return fail(c, rc);
  c->cur = 1 - c->cur;
  // 6. global records and measurements
  for (int p = 0; p < np; ++p) {
    StepRec& r = s->rec[p][(size_t)t];
    r = StepRec{};
    r.R_prev = (int32_t)s->R_glob[p];
    r.kmin_prev = loc[p].kmin_prev;
    r.culled = (int32_t)culled[p];
    r.S_prime = loc[p].S_prime;
    r.eps_expected = loc[p].eps_expected;
    r.S_t = c->sweeps[(size_t)t];
    s->R_glob[p] = R_new[p];
  }
  rc = shard_measure(s, t);
  if (rc != PA_OK) return fail(c, rc);
  c->t = t;
  c->stats.steps += 1;
  if (t == c->cfg.n_temps - 1) c->done = true;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_shard_observables(pa_shard* s, int32_t t, int32_t pop, pa_obs* out) try {
  if (!s || !out || t < 0 || pop < 0 || pop >= s->c->g.n_pop) return PA_ERR_INVALID;
  if (t > s->c->t) return PA_ERR_STATE;
  const StepRec* r0 = s->c->g.n_pop == 2 ? &s->rec[0][(size_t)t] : nullptr;
  pm1_observables(s->c->g, s->c->betas, s->rec[pop].data(), s->hist[pop].data() + (size_t)t * s->c->g.n_levels, t,
                  r0, out);
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_shard_local(pa_shard* s, pa_ctx** local) try {
  if (!s || !local) return PA_ERR_INVALID;
  *local = s->c;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_shard_extent(pa_shard* s, int32_t pop, int64_t* lo, int64_t* R_tilde) try {
  if (!s || pop < 0 || pop >= s->c->g.n_pop) return PA_ERR_INVALID;
  if (lo) *lo = s->lo;
  if (R_tilde) *R_tilde = s->R_glob[pop];
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_shard_q_hist(pa_shard* s, int32_t t, int64_t* out, int64_t cap) try {
  if (!s || !out || t < 0 || s->c->g.n_pop != 2) return PA_ERR_INVALID;
  if (t > s->c->t) return PA_ERR_STATE;
  if (cap < s->c->g.q_bins) return PA_ERR_CAPACITY;
  for (int i = 0; i < s->c->g.q_bins; ++i) out[i] = s->qhist[(size_t)t][(size_t)i];
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_shard_destroy(pa_shard* s) try {
  if (!s) return PA_ERR_INVALID;
  if (s->c) pa_destroy(s->c);
  if (s->dscratch) cudaFree(s->dscratch);
  if (s->dsizes) cudaFree(s->dsizes);
  delete s;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

}  // extern "C"

// ---------------------------------------------------------------- batch rounds
//
// The runs of a batch that qualify (+-1 couplings, an explicit schedule, a
// shared-memory sweep) advance together: a round takes each of them one step, as
// one reweighting launch for all their populations, one resampling launch, one
// sweep launch per (L, launch shape), one overlap launch for the two-population
// runs and a one-thread launch that advances the round counter.  Every launch
// reads its units' steps from device tables built here, so one CUDA graph,
// captured once, serves every round.  Each run's results are those of pa_step:
// the kernels of a round do for every unit what a lone run's launches do for it.

namespace pa {

struct Group {
  std::vector<pa_ctx*> runs;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<char> image;  // host copy of the device tables (kept until the copy is done)
  char* dev = nullptr;
  int32_t* round = nullptr;
  GroupUnit* units = nullptr;
  int32_t* res_off = nullptr;
  GroupPair* pairs = nullptr;
  int32_t* pair_off = nullptr;
  struct SweepLaunch {
    int L, shape, n, n_blocks;
    int32_t* list;
    int32_t* off;
  };
  std::vector<SweepLaunch> sweeps;
  int n_units = 0, res_blocks = 0, n_pairs = 0, pair_blocks = 0, max_levels = 0, max_bins = 0, n_rounds = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t launches_per_round = 0;
  // the sweeps of different (L, shape) are parallel branches of the round's graph
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
};

int64_t run_kernel_launches(const pa_ctx* c) { return c ? c->stats.kernel_launches : 0; }

bool group_eligible(const pa_ctx* c) {
  return c && c->model == PA_MODEL_PM1 && !c->adaptive && sweep_supported(c->g.L) && !c->g.shard &&
         c->error == PA_OK && !c->done;
}

void group_destroy(Group* G) {
  if (!G) return;
  if (G->stream) cudaStreamSynchronize(G->stream);
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->dev) cudaFreeAsync(G->dev, G->stream);
  if (G->stream) {
    cudaStreamSynchronize(G->stream);
    cudaStreamDestroy(G->stream);
  }
  if (G->ev) cudaEventDestroy(G->ev);
  for (cudaStream_t x : G->side) cudaStreamDestroy(x);
  for (cudaEvent_t e : G->join) cudaEventDestroy(e);
  delete G;
}

namespace {

// Offsets of the device tables within one allocation (16-byte aligned).
struct Layout {
  size_t bytes = 0;
  size_t take(size_t n) {
    const size_t at = (bytes + 15) & ~(size_t)15;
    bytes = at + n;
    return at;
  }
};

int group_build(Group* G) {
  const int n_runs = (int)G->runs.size();
  Layout lay;
  const size_t at_round = lay.take(sizeof(int32_t));
  std::vector<size_t> at_steps((size_t)n_runs);
  std::vector<int> first_unit((size_t)n_runs);
  for (int i = 0; i < n_runs; ++i) {
    const pa_ctx* c = G->runs[(size_t)i];
    at_steps[(size_t)i] = lay.take(sizeof(GroupStep) * (size_t)c->cfg.n_temps);
    first_unit[(size_t)i] = G->n_units;
    G->n_units += c->g.n_pop;
    if (c->g.n_pop == 2) ++G->n_pairs;
    G->max_levels = std::max(G->max_levels, c->g.n_levels);
    if (c->g.n_pop == 2) G->max_bins = std::max(G->max_bins, c->g.q_bins);
    G->n_rounds = std::max(G->n_rounds, c->cfg.n_temps - 1 - c->t);
  }
  const size_t at_units = lay.take(sizeof(GroupUnit) * (size_t)G->n_units);
  const size_t at_res = lay.take(sizeof(int32_t) * ((size_t)G->n_units + 1));
  const size_t at_pairs = lay.take(sizeof(GroupPair) * (size_t)std::max(G->n_pairs, 1));
  const size_t at_poff = lay.take(sizeof(int32_t) * ((size_t)G->n_pairs + 1));
  // sweep launches: the units of each (L, shape), in batch order
  std::map<std::pair<int, int>, std::vector<int32_t>> by_shape;
  for (int i = 0; i < n_runs; ++i) {
    const pa_ctx* c = G->runs[(size_t)i];
    for (int p = 0; p < c->g.n_pop; ++p) by_shape[{c->g.L, c->g.sweep_shape}].push_back(first_unit[(size_t)i] + p);
  }
  std::vector<std::pair<size_t, size_t>> at_sweep;
  for (const auto& kv : by_shape) {
    const size_t n = kv.second.size();
    at_sweep.emplace_back(lay.take(sizeof(int32_t) * n), lay.take(sizeof(int32_t) * (n + 1)));
  }
  G->image.assign(lay.bytes, 0);
  int rc = cuda_status(cudaMallocAsync(reinterpret_cast<void**>(&G->dev), lay.bytes, G->stream));
  if (rc != PA_OK) return rc;
  char* img = G->image.data();
  char* dev = G->dev;
  G->round = reinterpret_cast<int32_t*>(dev + at_round);
  G->units = reinterpret_cast<GroupUnit*>(dev + at_units);
  G->res_off = reinterpret_cast<int32_t*>(dev + at_res);
  G->pairs = reinterpret_cast<GroupPair*>(dev + at_pairs);
  G->pair_off = reinterpret_cast<int32_t*>(dev + at_poff);
  GroupUnit* units = reinterpret_cast<GroupUnit*>(img + at_units);
  int32_t* res_off = reinterpret_cast<int32_t*>(img + at_res);
  GroupPair* pairs = reinterpret_cast<GroupPair*>(img + at_pairs);
  int32_t* pair_off = reinterpret_cast<int32_t*>(img + at_poff);
  int k = 0, q = 0;
  res_off[0] = 0;
  pair_off[0] = 0;
  for (int i = 0; i < n_runs; ++i) {
    const pa_ctx* c = G->runs[(size_t)i];
    GroupStep* steps = reinterpret_cast<GroupStep*>(img + at_steps[(size_t)i]);
    for (int t = c->t + 1; t < c->cfg.n_temps; ++t) {
      const double dbeta = c->betas[(size_t)t] - c->betas[(size_t)t - 1];
      auto it = c->wtables.find(bits_of(dbeta));
      if (it == c->wtables.end()) return PA_ERR_INVALID;
      steps[t].w = it->second;
      metropolis_thresholds(c->betas[(size_t)t], steps[t].thr);
      steps[t].n_sweeps = c->sweeps[(size_t)t];
    }
    for (int p = 0; p < c->g.n_pop; ++p, ++k) {
      GroupUnit& u = units[k];
      u.g = c->g;
      u.P = c->pops[p];
      u.jtab = c->jtab;
      u.status = c->status;
      u.steps = reinterpret_cast<const GroupStep*>(dev + at_steps[(size_t)i]);
      u.t0 = c->t;
      u.cur0 = c->cur;
      u.last_t = c->cfg.n_temps - 1;
      u.pop = p;
      res_off[k + 1] = res_off[k] + (int32_t)((c->g.R_cap + kResampleSlotsPerBlock - 1) / kResampleSlotsPerBlock);
    }
    if (c->g.n_pop == 2) {
      pairs[q] = GroupPair{first_unit[(size_t)i], first_unit[(size_t)i] + 1, c->qhist};
      pair_off[q + 1] = pair_off[q] + (int32_t)((c->g.pitch / 4 + 255) / 256);
      ++q;
    }
  }
  G->res_blocks = res_off[G->n_units];
  G->pair_blocks = pair_off[G->n_pairs];
  size_t s = 0;
  for (const auto& kv : by_shape) {
    const int L = kv.first.first, shape = kv.first.second, tj = sweep_tile_slots(L, shape);
    if (tj <= 0) return PA_ERR_INVALID;
    const int n = (int)kv.second.size();
    int32_t* list = reinterpret_cast<int32_t*>(img + at_sweep[s].first);
    int32_t* off = reinterpret_cast<int32_t*>(img + at_sweep[s].second);
    off[0] = 0;
    for (int j = 0; j < n; ++j) {
      list[j] = kv.second[(size_t)j];
      off[j + 1] = off[j] + (int32_t)((units[list[j]].g.R_cap + tj - 1) / tj);
    }
    G->sweeps.push_back({L, shape, n, off[n], reinterpret_cast<int32_t*>(dev + at_sweep[s].first),
                         reinterpret_cast<int32_t*>(dev + at_sweep[s].second)});
    ++s;
  }
  return cuda_status(cudaMemcpyAsync(G->dev, img, lay.bytes, cudaMemcpyHostToDevice, G->stream));
}

// The launches of one round, captured into the group's graph: reweighting and
// resampling, then the sweeps of each (L, shape) as parallel branches (their last
// waves overlap), then the overlaps and the round counter.
int group_round(Group* G) {
  int rc = launch_rc(launch_group_reweight(G->units, G->n_units, G->max_levels, G->round, G->stream));
  if (rc == PA_OK)
    rc = launch_rc(launch_group_resample(G->units, G->res_off, G->n_units, G->res_blocks, G->round, G->stream));
  if (rc == PA_OK && !G->side.empty()) rc = cuda_status(cudaEventRecord(G->join[0], G->stream));
  for (size_t i = 0; i < G->sweeps.size() && rc == PA_OK; ++i) {
    const auto& sw = G->sweeps[i];
    cudaStream_t s = i == 0 ? G->stream : G->side[i - 1];
    if (i > 0) rc = cuda_status(cudaStreamWaitEvent(s, G->join[0], 0));
    if (rc == PA_OK)
      rc = launch_rc(launch_group_sweep(sw.L, sw.shape, G->units, sw.list, sw.off, sw.n, sw.n_blocks, G->round, s));
    if (rc == PA_OK && i > 0) rc = cuda_status(cudaEventRecord(G->join[i], s));
  }
  for (size_t i = 1; i < G->sweeps.size() && rc == PA_OK; ++i)
    rc = cuda_status(cudaStreamWaitEvent(G->stream, G->join[i], 0));
  if (rc == PA_OK && G->n_pairs > 0)
    rc = launch_rc(launch_group_overlap(G->units, G->pairs, G->pair_off, G->n_pairs, G->pair_blocks, G->max_bins,
                                        G->round, G->stream));
  if (rc == PA_OK) rc = launch_rc(launch_group_advance(G->round, G->stream));
  return rc;
}

}  // namespace

int group_create(pa_ctx* const* runs, int n, Group** out) {
  *out = nullptr;
  Group* G = new (std::nothrow) Group();
  if (!G) return PA_ERR_NOMEM;
  G->runs.assign(runs, runs + n);
  int rc = cuda_status(cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking));
  if (rc == PA_OK) rc = cuda_status(cudaEventCreateWithFlags(&G->ev, cudaEventDisableTiming));
  // the group starts after everything already issued on the runs' own streams
  for (pa_ctx* c : G->runs) {
    if (rc != PA_OK) break;
    rc = cuda_status(cudaEventRecord(G->ev, c->stream));
    if (rc == PA_OK) rc = cuda_status(cudaStreamWaitEvent(G->stream, G->ev, 0));
  }
  if (rc == PA_OK) rc = group_build(G);
  for (size_t i = 0; i < G->sweeps.size() && rc == PA_OK; ++i) {
    cudaEvent_t e = nullptr;
    rc = cuda_status(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (rc == PA_OK) G->join.push_back(e);
    if (rc == PA_OK && i > 0) {
      cudaStream_t x = nullptr;
      rc = cuda_status(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
      if (rc == PA_OK) G->side.push_back(x);
    }
  }
  // shared-memory limits of the sweep kernels are set before the capture
  for (const auto& sw : G->sweeps)
    if (rc == PA_OK)
      rc = launch_rc(launch_group_sweep(sw.L, sw.shape, G->units, sw.list, sw.off, sw.n, 0, G->round, G->stream));
  if (rc == PA_OK && G->n_rounds > 0) {
    cudaGraph_t graph = nullptr;
    rc = cuda_status(cudaStreamBeginCapture(G->stream, cudaStreamCaptureModeRelaxed));
    if (rc == PA_OK) {
      const int rr = group_round(G);
      const int re = cuda_status(cudaStreamEndCapture(G->stream, &graph));
      rc = rr != PA_OK ? rr : re;
    }
    if (rc == PA_OK) rc = cuda_status(cudaGraphInstantiate(&G->exec, graph, 0));
    if (graph) cudaGraphDestroy(graph);
    G->launches_per_round = 3 + (int64_t)G->sweeps.size() + (G->n_pairs > 0 ? 1 : 0);
  }
  if (rc != PA_OK) {
    group_destroy(G);
    return rc;
  }
  *out = G;
  return PA_OK;
}

int group_run(Group* G, int64_t* kernel_launches, int64_t* graph_launches) {
  int rc = PA_OK;
  for (int r = 0; r < G->n_rounds && rc == PA_OK; ++r) {
    rc = cuda_status(cudaGraphLaunch(G->exec, G->stream));
    if (rc == PA_OK) {
      *kernel_launches += G->launches_per_round;
      *graph_launches += 1;
    }
  }
  if (rc != PA_OK) return rc;
  // later work on a run's own stream (observables, further steps) follows the rounds
  rc = cuda_status(cudaEventRecord(G->ev, G->stream));
  for (pa_ctx* c : G->runs)
    if (rc == PA_OK) rc = cuda_status(cudaStreamWaitEvent(c->stream, G->ev, 0));
  if (rc != PA_OK) return rc;
  for (pa_ctx* c : G->runs) {
    const int k = c->cfg.n_temps - 1 - c->t;
    for (int t = c->t + 1; t <= c->t + k; ++t) c->counted_steps.emplace_back(t, c->sweeps[(size_t)t]);
    c->stats.steps += k;
    c->cur ^= (k & 1);
    c->t += k;
    c->done = true;
  }
  return PA_OK;
}

}  // namespace pa
