// pa_internal.h — structures shared by the host runtime (pa_runtime.cpp) and
// the kernels (pa_kernels.cu, pa_sweep.cu).  Plain C++ (no CUDA types) so the
// runtime can be compiled by the host compiler alone.
#pragma once
#include <cstddef>
#include <cstdint>

namespace pa {

// The status code of the C++ exception being handled, for the catch block of every
// entry point of the C interface (none lets an exception leave the library): a
// failed host allocation is PA_ERR_NOMEM, anything else PA_ERR_INVALID.
int exception_status() noexcept;

// Random-stream purposes (4 bits above the seed in the Philox key).
enum Purpose : uint32_t { kCouplings = 0, kInit = 1, kMetropolis = 2, kResample = 3 };

// Device status flags (OR-ed into one word by the kernels).
enum StatusFlag : int32_t { kFlagCapacity = 1, kFlagExtinct = 2, kFlagTimeout = 4 };

// Per-step, per-population record written by the kernels.
struct StepRec {
  int32_t R_tilde;      // population size after resampling into step t
  int32_t R_prev;       // population size of step t-1
  int32_t kmin_prev;    // lowest occupied level of step t-1
  int32_t culled;       // old replicas that received zero copies
  double S_prime;       // sum_k c_{t-1}(k) w(k - kmin)
  double eps_expected;  // (1/R) sum_k c(k) (1 - tau_k)_+
  unsigned long long sum_eta2;
  unsigned long long n_families;
  long long nll_hi;             // sum over families of nu ln nu (nu = eta / R~) as a 128-bit
  unsigned long long nll_lo;    // fixed-point number in units of 2^-100 (hi * 2^64 + lo), exact
  unsigned long long q_pairs;   // population 0 only
  unsigned long long q_small;   // population 0 only: pairs with 5|Q| <= N
  int32_t S_t;          // sweeps done at this step
  int32_t pad;
};

// Per-step, per-population record of the Gaussian-coupling model (energies in
// fixed point, units of 2^-20).
struct GRec {
  long long E_min;                 // lowest energy of the step-t population
  long long E0;                    // lowest energy over steps 0..t
  long long sum_E;                 // exact sum of energies
  unsigned long long sum_E2_lo;    // exact 128-bit sum of squared energies
  unsigned long long sum_E2_hi;
  long long n_at_E0;               // replicas at E0
  long long ql_sum;                // population 0: sum over pairs of the link-overlap bond sum
  long long pad;
};

// Device buffers of one population.
struct PopDev {
  int8_t* spins[2];     // [N][pitch] int8 +1/-1, site-major (replicas contiguous)
  int32_t* labels[2];   // [R_cap] family labels
  int32_t* levels;      // [pitch] energy level k of each slot of the current population
  int32_t* counts;      // [R_cap] copy numbers of the old slots
  int32_t* parents;     // [R_cap] parent (old slot) of each new slot
  int32_t* blocksums;   // [n_count_blocks] per-block copy totals, then their exclusive scan
  unsigned long long* tiles;  // [n_count_blocks] single-pass resampling: (2t+1 | 2t+2) << 32 | total or prefix
  int32_t* ticket;      // [1] single-pass resampling: next tile number (reset before each pass)
  uint32_t* hist;       // [n_temps][n_levels] energy-level histograms
  int32_t* fl;          // [n_levels] floor(tau_k)
  uint32_t* thr;        // [n_levels] 2^32 frac(tau_k)
  int32_t* mhist;       // [R_cap + 1] number of families of each size (filled on request)
  int32_t* fhist;       // [R_cap + 1] the running step's family sizes (zero between steps)
  int32_t* fsizes;      // [n_fsizes] the distinct sizes counted in fhist this step
  int32_t* fcount;      // [2] listed sizes, blocks done with this step's families (zero between steps)
  StepRec* rec;         // [n_temps]
  // Gaussian-coupling model only (null otherwise)
  long long* E64;       // [pitch] energies of the current population, units of 2^-20
  double* w;            // [R_cap] resampling weights of the old population
  double* part;         // [tree_sum_scratch(n_chunks)] fixed-order partial sums (chunks of 256 slots, then levels)
  int32_t* gfl;         // [R_cap] floor(tau_i)
  uint32_t* gthr;       // [R_cap] 2^32 frac(tau_i)
  unsigned long long* e2part;  // [2 * n_measure_blocks] 128-bit partial sums of E^2
  GRec* grec;           // [n_temps]
  uint32_t key_met[2];
  uint32_t key_res[2];
  uint32_t key_init[2];
};

// Geometry of one run.
struct RunGeom {
  int32_t L, N, n_levels;
  int64_t pitch;        // bytes per site row of the spin arrays (multiple of 1024)
  int32_t R;            // target population
  int32_t R_cap;
  int32_t n_pop;
  int32_t q_bins;
  int32_t n_count_blocks;    // resampling blocks (1024 slots each)
  int32_t n_fsizes;          // bound on the distinct family sizes of a population: floor(sqrt(2 R_cap)) + 2
  int32_t sweep_shape;       // index of the sweep kernel's launch shape among those of L
  // A run of a single GPU whose last wave of sweep tiles would be mostly empty sweeps
  // the slots from tail_from on (a multiple of 1024) with the smaller tiles of shape
  // tail_shape, spread over the SMs, in a second launch (-1: one launch).
  int32_t tail_shape;
  int32_t tail_from;
  int32_t model;             // 0: +-1 couplings, 1: Gaussian couplings (fixed point)
  // One rank's share of a sharded population (pa_shard): global slot of local slot
  // 0 (a multiple of 1024; random words are addressed by global slot), the local
  // initial population, and whether the sweep leaves the family statistics to the
  // sharded step (families may straddle ranks).  0, R, 0 for a whole population.
  int32_t slot_base;
  int32_t n_init;
  int32_t shard;
  int32_t n_chunks;          // Gaussian: chunks of 256 slots of the weight sums
  int32_t n_measure_blocks;  // Gaussian: blocks of the energy-moment reduction
};

// Acceptance table of a site (Gaussian model): for each of the 64 patterns of
// antiparallel neighbours (bit k: bond k, in the order x+1, x-1, y+1, y-1, z+1,
// z-1), the Metropolis threshold of flipping the site: 0xFFFFFFFF when the flip
// costs dE <= 0 (always taken), else min(floor(2^32 exp(-beta dE)), 2^32 - 2).
constexpr int kGPatterns = 64;

constexpr int kChunk = 256;            // slots per fixed-order partial sum (Gaussian weights)
// Entries of the Gaussian partial-sum buffer for n chunk totals: the totals, then
// the outputs of every level of the fixed-order tree but the last.
inline int64_t tree_sum_scratch(int64_t n) {
  int64_t total = n;
  for (int64_t m = n; m > kChunk;) {
    m = (m + kChunk - 1) / kChunk;
    total += m;
  }
  return total;
}
constexpr int kGTableWeights = 16384;  // doubles per step: weight tables T0 | T1 | T2

// One launch shape of the sweep kernel (every shape gives identical results).
struct SweepShapeInfo {
  int32_t L, W, NT, MB;  // lattice size, words per site row, threads per CTA, CTAs per SM compiled for
  int32_t smem;          // dynamic shared memory per CTA, bytes
};
int sweep_shape_count(int L);
bool sweep_shape_info(int L, int i, SweepShapeInfo* out);
// The tail launch of a run of target population R with main shape `shape` on a
// device of n_sm SMs: sets *tail_shape and *tail_from, or *tail_shape = -1 when one
// launch is as good (its last wave is full enough, or L has no smaller tile).
void sweep_tail_plan(int L, int shape, int64_t R, int n_sm, int32_t* tail_shape, int32_t* tail_from);

constexpr int kCountThreads = 256;     // threads per resampling block
constexpr int kSlotsPerCountBlock = 1024;

// ---- launchers (pa_kernels.cu / pa_sweep.cu); each returns a cudaError_t as int ----
int launch_init_couplings(const RunGeom& g, uint64_t disorder_seed, int8_t* J, uint32_t* jtab, void* stream);
int launch_init_population(const RunGeom& g, PopDev* pops, int cur, void* stream);
int launch_levels_and_hist(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, int t, void* stream);
int launch_reweight(const RunGeom& g, PopDev* pops, const double* w, int t, void* stream);
// Polls after which a look-back wait of the single-pass resampling gives up.
constexpr int kLookbackSpins = 1 << 20;
// Test setting of that wait: the poll limit (0: kLookbackSpins) and a tile whose
// block publishes nothing (-1: none).
struct LookbackTest {
  int32_t spins = 0;
  int32_t withheld_tile = -1;
};
// Single-pass resampling of the +-1 model; launch_reweight of the same step, on the
// same stream just before, resets the tile ticket it relies on.
int launch_resample(const RunGeom& g, PopDev* pops, int cur, int t, int32_t* status, const LookbackTest& test,
                    void* stream);
int launch_sweep(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, int t, int n_sweeps,
                 const uint32_t met_thr[3], void* stream);
// Family statistics of step t (sum of eta^2, families, sum of nu ln nu) into the step
// records; the +-1 shared-memory sweep does the same in its epilogue.
int launch_families(const RunGeom& g, PopDev* pops, int cur, int t, void* stream);
// The family-size histogram m(eta) of population pop at step t into its mhist
// (on request: the step records are not touched).
int launch_family_hist(const RunGeom& g, PopDev* pops, int pop, int cur, int t, void* stream);
// Gaussian-coupling model (pa_gauss.cu, and k_sweep_g in pa_sweep.cu)
int launch_scan_scatter(const RunGeom& g, PopDev* pops, int cur, int t, int32_t* status, void* stream);
int launch_g_energy_init(const RunGeom& g, PopDev* pops, int cur, const int32_t* Jq, void* stream);
int launch_g_resample(const RunGeom& g, PopDev* pops, int cur, int t, const double* wtab, int32_t* status,
                      void* stream);
int launch_g_sweep(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, const int32_t* Jq, long long Jtot,
                   const uint32_t* gtab, int t, int n_sweeps, void* stream);
// The expected culling fraction of population 0 for the weight tables wtab, into
// rec[t].eps_expected (also overwrites the step-t weights, sums and tables, which the
// resampling recomputes): one evaluation of the adaptive bisection.
int launch_g_eps_trial(const RunGeom& g, PopDev* pops, int t, const double* wtab, void* stream);
int launch_g_measure(const RunGeom& g, PopDev* pops, int cur, int t, unsigned long long* qlhist, void* stream);
// Weight tables of dbeta (*dbeta_dev, or dbeta_val when it is null) built on the device.
int launch_g_tables(const double* dbeta_dev, double dbeta_val, double* T, void* stream);
// `halvings` halvings of the adaptive bisection on the device, with no host wait:
// b = {lo, hi, mid, 0} in device memory; each halving builds mid's tables in T, runs
// the trial of launch_g_eps_trial and updates b, until b[3] marks the fixed point
// (mid equal to a point already decided), after which the halvings do no work.
int launch_g_bisect(const RunGeom& g, PopDev* pops, int t, double* T, double* b, double target, int halvings,
                    void* stream);
// The same halvings in one cooperative launch of n_blocks blocks (g_bisect_blocks:
// 0 when the device or the population size does not allow it): tables = three sets
// of kGTableWeights entries, part1 = n_chunks partial sums, bar = 8 words (barrier
// and totals, cleared on the stream first).  On return b = {lo, hi, mid, state}, state -1 when
// a grid barrier wait ran out (the interval is then not to be used).  withheld >= 0 (tests):
// that block does not arrive at the first barrier and the waits poll 4096 times, so they run out.
int g_bisect_blocks(const RunGeom& g);
int launch_g_bisect_fused(const RunGeom& g, PopDev* pops, int t, double* tables, double* part1,
                          unsigned long long* bar, double* b, double target, int halvings, int n_blocks,
                          int withheld, void* stream);
int launch_overlap(const RunGeom& g, PopDev* pops, int cur, int t, unsigned long long* qhist, void* stream);

// ---- a batch advanced by one launch per kernel and temperature step (pa_batch) ----
// Every population of every run of the batch is a unit; a round takes each unit's
// run one step further with one reweighting launch, one resampling launch, one
// sweep launch per (L, launch shape) and one overlap launch, all reading the round
// number from device memory, so the same CUDA graph serves every round.  In round
// r a unit's step is t = t0 + 1 + r (the unit rests once t > last_t) and the
// population it reads is buffer cur0 ^ (r & 1).
struct GroupStep {   // step t of a run (t >= 1)
  const double* w;   // the run's weight table of beta_t - beta_{t-1} (device)
  uint32_t thr[3];   // Metropolis thresholds of beta_t for dE = 4, 8, 12
  int32_t n_sweeps;
};
struct GroupUnit {   // one population of one run
  RunGeom g;
  PopDev P;
  const uint32_t* jtab;
  int32_t* status;
  const GroupStep* steps;  // [n_temps], entry 0 unused
  int32_t t0, cur0, last_t, pop;
};
struct GroupPair {   // the two populations of a two-population run
  int32_t u0, u1;
  unsigned long long* qhist;
};
// Block ranges: units (or pairs) k take the blocks [off[k], off[k + 1]) of a launch.
int launch_group_reweight(const GroupUnit* units, int n_units, int max_levels, const int32_t* round, void* stream);
int launch_group_resample(const GroupUnit* units, const int32_t* off, int n_units, int n_blocks,
                          const int32_t* round, void* stream);
// Sweep of the units list[0, n) (all of lattice size L and launch shape `shape`),
// off[k] = first tile of unit list[k] in the launch.
int launch_group_sweep(int L, int shape, const GroupUnit* units, const int32_t* list, const int32_t* off, int n,
                       int n_blocks, const int32_t* round, void* stream);
int launch_group_overlap(const GroupUnit* units, const GroupPair* pairs, const int32_t* off, int n_pairs,
                         int n_blocks, int max_bins, const int32_t* round, void* stream);
int launch_group_advance(int32_t* round, void* stream);
// Tiles (slots per CTA) of sweep shape `shape` of L; 0 if there is none.
int sweep_tile_slots(int L, int shape);
constexpr int kResampleSlotsPerBlock = 1024;  // old slots per block of the single-pass resampling

}  // namespace pa
struct pa_ctx;
namespace pa {
// A run created for overlapped execution keeps the device's chosen sweep shape
// (no switch to smaller tiles for a small population).
void use_chosen_shape(pa_ctx* c);
#ifdef PA_H
// pa_create, optionally without its final stream synchronisation (a Gaussian run
// always synchronises, its host tables being temporaries): for runs created among
// many others (pa_batch, pa_server), whose next synchronisation reports any error
// of the initialisation.
int create_run(const pa_config* cfg, void* cuda_stream, pa_ctx** out, bool synchronize);
// The same for one rank's share of a sharded run: the global slots
// [slot_base, slot_base + n_init) of the initial population (slot_base a multiple
// of 1024), family statistics left to the sharded step.
int create_run_share(const pa_config* cfg, void* cuda_stream, pa_ctx** out, int64_t slot_base, int64_t n_init);
#endif
// Batch rounds (pa_batch): the runs that qualify (+-1 couplings, explicit schedule,
// shared-memory sweep, not finished) advance together, one CUDA graph launch per
// round; group_run issues every round (asynchronously), makes the runs' streams wait
// for them and advances the runs' host state to their last step.
struct Group;
bool group_eligible(const pa_ctx* c);
int group_create(pa_ctx* const* runs, int n, Group** out);
int group_run(Group* grp, int64_t* kernel_launches, int64_t* graph_launches);
void group_destroy(Group* grp);
// Kernel launches a run has issued (its pa_stats count, without synchronising).
int64_t run_kernel_launches(const pa_ctx* c);
// Largest lattice size the sweep kernel supports.
constexpr int kMaxL = 16;
// Largest lattice size of a run (larger lattices than kMaxL sweep in global memory).
constexpr int kMaxLGlobal = 64;
bool sweep_supported(int L);        // shared-memory sweep kernels (even L <= kMaxL)
bool lattice_supported(int L);      // every lattice a run accepts (even L <= kMaxLGlobal)
// Global-memory sweep for kMaxL < L <= kMaxLGlobal (pa_sweep_global.cu): replica copy,
// S half-sweep launches in place, energy levels.
int launch_sweep_global(const RunGeom& g, PopDev* pops, int cur, const uint32_t* jtab, int t, int n_sweeps,
                        const uint32_t met_thr[3], void* stream);
// Sharded runs: the copies of population pop's resampling written out as replicas,
// new[n][j] = old[n][parents[j]] for j < rec[t].R_tilde (pa_sweep_global.cu).
int launch_copy_parents(const RunGeom& g, PopDev* pops, int pop, int cur, int t, void* stream);
// Family runs of one rank's slots (labels[cur][0, rec[t].R_tilde)): the first and
// the last run (they may continue on other ranks) into edge = {has slots, first
// label, first length, last label, last length, runs, sum of eta^2 and number of
// the other runs}, the other runs also into mhist (which starts at zero).
int launch_shard_families(const RunGeom& g, PopDev* pops, int pop, int cur, int t, long long* edge, void* stream);
// The sum over the sizes eta[k] (m[k] families each, k < K) of m nu ln nu,
// nu = eta / R_new, exactly as the step's family statistics add it, into
// out = {hi, lo} (pa_family.cuh).
int launch_entropy_of_sizes(const int32_t* eta, const int32_t* m, int K, int R_new, long long* out, void* stream);

}  // namespace pa
