/* pa.h — C ABI of the GB300 population annealing library (libpa.so).
 *
 * Population annealing (PA) as defined by Amey & Machta, "Analysis and
 * Optimization of Population Annealing" (§II): a population of R replicas of a
 * 3D Edwards-Anderson spin glass (L^3 sites, periodic, +-1 couplings J_nm) is
 * cooled from beta = 0 through a schedule beta_0 < beta_1 < ...; each step
 *   1. resamples beta_{t-1} -> beta_t: replica i gets n_i copies with
 *      E n_i = tau_i = (R / R~) exp(-(beta_t - beta_{t-1}) E_i) / Q   (Eqs. tau, Q)
 *      by the nearest-integer rule (n_i = floor or ceil of tau_i),
 *   2. runs S_t checkerboard Metropolis sweeps at beta_t,
 *   3. measures the estimators of §II.A and §III.A: energy moments, the free
 *      energy -beta F~ (Eq. betaF), ground-state estimators (Eq. g0), family
 *      statistics rho_t (Eq. rho_t_def2) and the family entropy, and the spin
 *      overlap q histogram of two independent populations.
 * The temperature schedule is either given, or chosen step by step to hold the
 * expected culling fraction of Eq. (eq_num_elim) at a target (§IV.B).
 *
 * Every step of the path runs in CUDA kernels for sm_103a on the stream given
 * at creation.  All pointers in this header are HOST pointers unless stated
 * otherwise.  Functions never throw; they return a status code.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by (seed, purpose,
 * population) and countered by (site, sweep, slot, step), so every result is a
 * deterministic function of the configuration, independent of launch shapes.
 *
 * Conventions: site n = x + L (y + L z); bond (n, d) joins n and n + e_d; the
 * energy level of a replica is k = (E + 3N) / 2 = its number of unsatisfied
 * bonds; step t = 0 is beta = 0 (the paper indexes the schedule downwards).
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PA_OK 0
#define PA_DONE 1            /* pa_step: the schedule is complete, nothing was done */
#define PA_ERR_INVALID (-1)  /* bad argument or configuration */
#define PA_ERR_NOMEM (-2)    /* device or host allocation failed (no C++ exception leaves the library) */
#define PA_ERR_CAPACITY (-3) /* population outgrew R_cap (detected on the device; nothing written out of bounds) */
#define PA_ERR_TIMEOUT (-4)  /* a bounded device wait gave up */
#define PA_ERR_CUDA (-5)     /* a CUDA runtime call failed */
#define PA_ERR_STATE (-6)    /* call out of order, e.g. a step that has not run yet */
#define PA_ERR_EXTINCT (-7)  /* every replica received zero copies */

/* ---- configuration of one run (§II; schedule §IV.B) ----
 * L            lattice size; even, 2 <= L <= 64 (up to 16 a CTA holds a tile of
 *              replicas in shared memory for all sweeps of a step; beyond, the
 *              sweeps run in global memory, one launch per half-sweep; Gaussian
 *              couplings up to 16).
 * n_pop        1, or 2 independent populations on the same couplings (for q).
 * R            target population size, 1 <= R.
 * R_cap        hard capacity of the population arrays (0 = R + 10 ceil(sqrt R) + 1024);
 *              R <= R_cap < 2^31.
 * disorder_seed, run_seed   < 2^56; couplings come from disorder_seed, spins,
 *              Metropolis and resampling from run_seed (population index in the key).
 * n_temps, betas  explicit schedule betas[0..n_temps) ascending with betas[0] = 0;
 *              or betas = NULL for the adaptive schedule, with n_temps the step
 *              limit, beta_max the last temperature and eps_target in (0,1) the
 *              culling fraction to hold.
 * n_sweeps, sweeps_per_step   sweeps of step t: sweeps_per_step[t] if non-NULL
 *              (n_temps entries), else n_sweeps.  Step 0 never sweeps.
 * q_bins       overlap histogram bins over q in [-1, 1] (odd, >= 3; 65 typical).
 * model        PA_MODEL_PM1: couplings +-1 with p = 1/2; PA_MODEL_GAUSS: couplings
 *              ~ N(0,1) (the paper's model, §II.A), clamped to [-5, 5] and held in
 *              fixed point (units of 2^-20), explicit schedules only.
 * The configuration and the arrays it points to are copied by pa_create. */
#define PA_MODEL_PM1 0
#define PA_MODEL_GAUSS 1
typedef struct {
  int32_t L;
  int32_t n_pop;
  int64_t R;
  int64_t R_cap;
  uint64_t disorder_seed;
  uint64_t run_seed;
  int32_t n_temps;
  const double* betas;
  double beta_max;
  double eps_target;
  int32_t n_sweeps;
  const int32_t* sweeps_per_step;
  int32_t q_bins;
  int32_t model;
} pa_config;

/* ---- observables of one population at step t (after the sweeps at beta_t) ----
 * The resampling fields describe the move beta_{t-1} -> beta_t (zero at t = 0). */
typedef struct {
  int32_t t;
  double beta, dbeta;
  int64_t R_tilde;        /* population size R~_t */
  int64_t sum_E, sum_E2;  /* exact sums of E and E^2 over the population */
  int32_t E_min;          /* lowest energy in the population */
  double mean_E, var_E;   /* population mean and variance of E */
  int32_t kmin_prev;      /* lowest level of the step t-1 population */
  double S_prime;         /* sum_i exp(-dbeta (E_i - E_min)) over the step t-1 population */
  double lnQ;             /* ln Q(beta_{t-1}, beta_t), Eq. (Q) */
  double minus_beta_F;    /* -beta_t F~(beta_t), Eq. (betaF) */
  double eps_expected;    /* expected culling fraction, Eq. (eq_num_elim) / R */
  int64_t culled;         /* replicas of step t-1 that received zero copies */
  int64_t sum_eta2;       /* sum over families of eta^2 */
  int64_t n_families;     /* families with at least one member */
  double rho_t;           /* sum eta^2 / R~_t */
  double S_f;             /* family entropy -sum nu ln nu, nu = eta / R~_t */
  double rho_s;           /* R~_t / exp(S_f) */
  int32_t E0;             /* lowest energy measured at steps 0..t */
  double g0_tilde;        /* fraction of the population at E0 */
  double g0_bar;          /* 2 exp(-beta E0 + beta F~), Eq. (g0) */
  int64_t q_pairs;        /* overlap pairs (slot j of population 0 with slot j of 1) */
  int64_t q_abs_le_02;    /* pairs with |q| <= 0.2 */
  double I02;             /* q_abs_le_02 / q_pairs, the per-sample I(0.2) */
} pa_obs;

/* ---- observables of a Gaussian-coupling run (model PA_MODEL_GAUSS) ----
 * Energies are exact integers in units of 2^-20; mean_E, var_E and the derived
 * quantities are in units of J.  The link overlap q_l (Eq. ql) is measured between
 * slot j of the two populations, with e_l (Eq. el) and e_l - <E>/N, the
 * per-sample term of Delta_KY (Eq. KY; its disorder average vanishes for
 * Gaussian couplings in equilibrium). */
typedef struct {
  int32_t t;
  double beta, dbeta;
  int64_t R_tilde;
  int64_t sum_E;          /* exact sum of E (units of 2^-20) */
  double sum_E2;          /* exact sum of E^2 (units of 2^-40), rounded once to double */
  int64_t E_min;          /* lowest energy at t */
  double mean_E, var_E;
  int64_t E_min_prev;     /* lowest energy of the step t-1 population */
  double S_prime, lnQ, minus_beta_F, eps_expected;
  int64_t culled, sum_eta2, n_families;
  double rho_t, S_f, rho_s;
  int64_t E0;             /* lowest energy at steps 0..t */
  double g0_tilde, g0_bar;
  int64_t q_pairs, q_abs_le_02;
  double I02;
  int64_t ql_sum;         /* sum over pairs of sum over bonds s1_n s1_m s2_n s2_m */
  double ql_mean;         /* <q_l> = ql_sum / (3N q_pairs) */
  double e_l;             /* -3 beta (1 - <q_l>) */
  double delta_KY;        /* e_l - <E>/N */
} pa_gobs;

typedef struct pa_ctx pa_ctx;

/* Creates a run: allocates its device memory (owned by the context; one
 * stream-ordered allocation of pa_footprint bytes, carved into the run's
 * buffers), draws the couplings and the initial population (uniform spins,
 * label = slot) with kernels on `cuda_stream` (a cudaStream_t; NULL = the legacy
 * default stream) and measures step 0.  Returns PA_OK and *out, or an error (and
 * *out = NULL; PA_ERR_NOMEM when the allocation fails). */
int pa_create(const pa_config* cfg, void* cuda_stream, pa_ctx** out);

/* Runs the next temperature step (resample, sweep, measure).  Asynchronous for
 * an explicit schedule; the adaptive schedule reads the previous energy
 * histogram back to the host to choose beta_t.  Returns PA_OK, PA_DONE when the
 * schedule is complete, or an error recorded by an earlier step. */
int pa_step(pa_ctx* ctx);

/* Runs all remaining steps and synchronises; returns PA_OK or the first error. */
int pa_run(pa_ctx* ctx);

/* Index of the last step run (0 right after pa_create). */
int32_t pa_current_step(const pa_ctx* ctx);

/* Fills *out for step t <= pa_current_step and population pop (+-1 couplings; the
 * Gaussian model: pa_gobservables).  Waits until step t is done, not for steps
 * issued after it: a caller may issue step t + 1 with pa_step and then read step t
 * while the GPU runs.  An error recorded on the device by then (capacity,
 * extinction, timeout) is returned; one of a later step is reported by a later call
 * (pa_sync waits for everything).  Reads step t's records and energy histogram from
 * the device (about 88 (t + 1) + 4 (3N + 1) bytes). */
int pa_observables(pa_ctx* ctx, int32_t t, int32_t pop, pa_obs* out);

/* Energy-level histogram c_t(k), k = 0..3N, of population pop at step t
 * (out: 3N+1 int64 entries; cap = capacity of out in entries). */
int pa_energy_hist(pa_ctx* ctx, int32_t t, int32_t pop, int64_t* out, int64_t cap);

/* Overlap histogram of step t: bin b = ((Q + N)(q_bins - 1) + N) div 2N of
 * Q = sum_n s^0_n s^1_n (two populations only; out: q_bins int64 entries). */
int pa_q_hist(pa_ctx* ctx, int32_t t, int64_t* out, int64_t cap);

/* Family-size histogram of the current population: *n pairs (eta[i], m[i]),
 * eta ascending, m[i] = number of families of size eta[i].  Returns
 * PA_ERR_CAPACITY (with *n set) if cap is too small. */
int pa_family_hist(pa_ctx* ctx, int32_t pop, int64_t cap, int64_t* eta, int64_t* m, int64_t* n);

/* Population size of pop at the current step. */
int pa_population_size(pa_ctx* ctx, int32_t pop, int64_t* count);

/* Copies slots [first, first + n) of population pop: spins replica-major
 * [n][N] int8 (+1/-1), family labels and energies E (each may be NULL). */
int pa_get_replicas(pa_ctx* ctx, int32_t pop, int64_t first, int64_t n, int8_t* spins, int32_t* labels,
                    int32_t* energies);

/* Copy numbers n_i of the old slots in the last resampling (*count = R~_{t-1})
 * and the parent (old slot) of every new slot (*count = R~_t).  PA_ERR_STATE at step 0. */
int pa_get_copy_counts(pa_ctx* ctx, int32_t pop, int32_t* counts, int64_t cap, int64_t* count);
int pa_get_parents(pa_ctx* ctx, int32_t pop, int32_t* parents, int64_t cap, int64_t* count);

/* Couplings J[3n + d] = +1/-1 (3N int8 entries). */
int pa_get_couplings(pa_ctx* ctx, int8_t* J, int64_t cap);

/* Inverse temperature of step t (t <= pa_current_step), or a negative value. */
double pa_beta(const pa_ctx* ctx, int32_t t);

/* ---- Gaussian-coupling runs (model PA_MODEL_GAUSS) ----
 * pa_observables, pa_energy_hist and the energies of pa_get_replicas are for
 * +-1 runs (PA_ERR_INVALID otherwise); a Gaussian run reads its observables,
 * energies, link-overlap histogram and couplings here. */
int pa_gobservables(pa_ctx* ctx, int32_t t, int32_t pop, pa_gobs* out);
/* Energies (units of 2^-20) of slots [first, first + n) of population pop. */
int pa_get_genergies(pa_ctx* ctx, int32_t pop, int64_t first, int64_t n, int64_t* E);
/* Link-overlap histogram of step t: bin ((Q_l + 3N)(q_bins - 1) + 3N) div 6N of
 * Q_l = sum over bonds s1_n s1_m s2_n s2_m; q_bins entries (two populations). */
int pa_ql_hist(pa_ctx* ctx, int32_t t, int64_t* out, int64_t cap);
/* Fixed-point couplings Jq[3n + d] (3N int32, units of 2^-20) of a Gaussian run. */
int pa_get_gcouplings(pa_ctx* ctx, int32_t* Jq, int64_t cap);

/* ---- instrumentation ----
 * Counters since the last pa_stats_reset: steps run, kernels launched by the
 * library, bytes copied host->device and device->host (by this context), and,
 * when timing is enabled, device time per phase measured with CUDA events
 * recorded on the run's stream around each phase of every step:
 *   PA_PHASE_REWEIGHT  Boltzmann reweighting tables (one block per population)
 *   PA_PHASE_RESAMPLE  copy numbers, scan, parents and labels
 *   PA_PHASE_SWEEP     parent gather + Metropolis sweeps + energy levels
 *   PA_PHASE_FAMILY    family sizes, sum eta^2, family entropy
 *   PA_PHASE_OVERLAP   overlap histogram (two populations only)
 * pa_get_stats synchronises the stream. */
#define PA_PHASE_REWEIGHT 0
#define PA_PHASE_RESAMPLE 1
#define PA_PHASE_SWEEP 2
#define PA_PHASE_FAMILY 3
#define PA_PHASE_OVERLAP 4
#define PA_N_PHASES 5
typedef struct {
  int64_t steps;
  int64_t kernel_launches;
  int64_t h2d_bytes;
  int64_t d2h_bytes;
  int64_t updates;                 /* Metropolis site updates: sum over steps of S_t N R~_t */
  double phase_ms[PA_N_PHASES];    /* summed device time per phase (timing enabled) */
  int64_t phase_count[PA_N_PHASES];/* timed launches of each phase */
} pa_stats;
int pa_stats_reset(pa_ctx* ctx, int enable_timing);
int pa_get_stats(pa_ctx* ctx, pa_stats* out);

/* ---- one population split across ranks (§I: PA runs on computing clusters) ----
 * A sharded run splits each population by slot across n_ranks processes: rank r
 * holds the global slots [lo_r, hi_r) of every population, whole units of 1024
 * slots as balanced as units allow (the last units of the population size), cut
 * from the larger population of the step so that slot j of both populations is
 * on one rank.  Every random word is addressed by global slot, so the results are
 * those of one process bit for bit (+-1 couplings, explicit schedules, even
 * L <= 16).  A temperature step (pa_shard_step, collective over all ranks):
 *   1. the level histogram of the last step is summed over ranks (allreduce), so
 *      every rank builds the same reweighting tables (Eqs. tau, Q);
 *   2. copy numbers of the local old slots; their totals are gathered from all
 *      ranks (allgather), which places each rank's copies in the global order;
 *   3. every copy moves to the rank that holds its new slot (send / recv, each pair
 *      of ranks in rank order: spins as N rows of bytes, then labels);
 *   4. sweeps of the local slots, local level histograms;
 *   5. measurements: histograms summed over ranks; families as runs of the sorted
 *      labels, the first and last run of every rank joined across rank
 *      boundaries; the overlap histogram of co-located slot pairs summed.
 * The host functions in pa_comm carry the exchanges (for example over gloo); each
 * returns 0 on success.  The runs of all ranks run on one device or several. */
typedef struct {
  void* user;
  /* element-wise sum over the ranks of n int64 values, in place */
  int (*allreduce_i64)(void* user, int64_t* values, int64_t n);
  /* n int64 values from every rank: out[q n + i] is value i of rank q */
  int (*allgather_i64)(void* user, const int64_t* values, int64_t n, int64_t* out);
  /* blocking point-to-point transfer of `bytes` bytes to / from another rank */
  int (*send)(void* user, int32_t dst, const void* buf, int64_t bytes);
  int (*recv)(void* user, int32_t src, void* buf, int64_t bytes);
} pa_comm;
typedef struct pa_shard pa_shard;

/* Rank `rank` of n_ranks (collective: all ranks call it with the same config).
 * The rank's device buffers are sized for the whole capacity R_cap (a rank may
 * receive every copy).  PA_ERR_INVALID for an adaptive schedule, Gaussian
 * couplings, L outside the shared-memory sweep or a bad rank. */
int pa_shard_create(const pa_config* cfg, int32_t rank, int32_t n_ranks, const pa_comm* comm, void* cuda_stream,
                    pa_shard** out);
/* One temperature step of every rank (collective); PA_DONE after the last. */
int pa_shard_step(pa_shard* shard);
/* Observables of step t (the whole population's, the same on every rank). */
int pa_shard_observables(pa_shard* shard, int32_t t, int32_t pop, pa_obs* out);
/* This rank's run (its slots of the current population), for the per-rank
 * readers (pa_get_replicas, pa_population_size, pa_get_copy_counts ...); it
 * belongs to the shard. */
int pa_shard_local(pa_shard* shard, pa_ctx** local);
/* Global slot of this rank's first slot, and the global population size. */
int pa_shard_extent(pa_shard* shard, int32_t pop, int64_t* lo, int64_t* R_tilde);
/* The overlap histogram of step t (q_bins entries, summed over the ranks). */
int pa_shard_q_hist(pa_shard* shard, int32_t t, int64_t* out, int64_t cap);
int pa_shard_destroy(pa_shard* shard);

/* ---- testing hook: the bounded wait of the resampling (§II, +-1 couplings) ----
 * The single-pass resampling finds each tile's offset by waiting, with a bounded
 * number of polls, for the entries its predecessor tiles publish.  This sets, for
 * the later steps of run ctx, that number of polls (spins >= 1; 0 restores the
 * default of 2^20) and a tile (numbered in the order its block starts) whose block
 * publishes neither its total nor its offset (withheld_tile >= 0; -1: none), so
 * that the waits of the blocks after it run out.  A wait that runs out ends the
 * kernel normally with the device timeout flag set: that step's results are not
 * valid, and the run reports PA_ERR_TIMEOUT from its next synchronising call
 * (pa_sync, pa_observables, ...) and every call after it.  The device, and other
 * runs on it, are not affected.  For tests of that failure path only;
 * PA_ERR_INVALID for spins < 0 or withheld_tile < -1. */
int pa_debug_lookback(pa_ctx* ctx, int32_t spins, int32_t withheld_tile);

/* ---- testing hook: the adaptive bisection of a Gaussian-coupling run (§IV.B) ----
 * Its halvings run in one cooperative launch where the device allows it
 * (one_launch = 1, the default) or as a few launches per halving (one_launch = 0);
 * both take the same decisions from the same sums, so the temperatures and every
 * result are the same.  In the one-launch form the blocks meet at grid barriers
 * whose waits poll a bounded number of times; withheld_block >= 0 keeps that block
 * (of the launch's blocks, numbered from 0; a number past the last keeps none) from
 * arriving at the first barrier and lowers the poll limit to 4096, so that the
 * others' waits run out: the launch then ends normally with its error set, and the
 * run reports PA_ERR_TIMEOUT from that step on.  The device and other runs on it are
 * not affected.  -1: none.  For tests only; PA_ERR_INVALID for a run without Gaussian
 * couplings or an adaptive schedule, one_launch outside {0, 1}, withheld_block < -1,
 * or withheld_block >= 0 with one_launch = 0. */
int pa_debug_bisect(pa_ctx* ctx, int32_t one_launch, int32_t withheld_block);

/* Waits for the context's stream; returns the first recorded error, if any. */
int pa_sync(pa_ctx* ctx);

/* Frees the context and its device memory (synchronises first). */
int pa_destroy(pa_ctx* ctx);

/* Static description of a status code. */
const char* pa_strerror(int status);

/* ---- many runs at once (batched and served workloads) ----
 * Independent runs (different couplings, sizes, populations, schedules) share
 * the GPU.  A batch advances its runs in rounds of one temperature step each (see
 * pa_batch_set_mode); the server runs each admitted run on its own non-blocking
 * stream, issuing steps round-robin from the host, so that the kernels of
 * different runs overlap on the device.  Each run gives exactly the results it
 * gives alone (its random streams depend only on its configuration).  These
 * objects are not thread-safe. */

/* Device bytes that pa_create allocates for cfg, exactly (for admission control;
 * no device call). */
int pa_footprint(const pa_config* cfg, size_t* bytes);

typedef struct pa_batch pa_batch;
/* Creates n runs (configs copied), each on its own stream. */
int pa_batch_create(const pa_config* cfgs, int32_t n, pa_batch** out);
/* Advances every run to the end of its schedule, one step of each run per
 * round, then synchronises; returns PA_OK or the first error.  A run that fails
 * (its own status, see pa_sync) stops there; the other runs still finish. */
int pa_batch_run(pa_batch* batch);

/* How pa_batch_run advances the runs (both give every run its results alone):
 * PA_BATCH_FUSED (the default): the runs that qualify — +-1 couplings, an
 *   explicit schedule, L <= 16, not finished — advance together, each round one
 *   reweighting launch for all their populations, one resampling launch, one sweep
 *   launch per lattice size and launch shape, one overlap launch for the
 *   two-population runs and a one-thread launch that advances the device's round
 *   counter.  The round reads each run's step (its weight table, Metropolis
 *   thresholds and sweeps) from device tables built when pa_batch_run starts, so
 *   the launches of one round are captured once as a CUDA graph and every round is
 *   one graph launch, all issued without waiting; runs that finish earlier rest in
 *   the later rounds.  The other runs step on their own streams as below.
 * PA_BATCH_STREAMS: every run steps on its own stream, one pa_step of each run per
 *   round, issued from the host.
 * PA_ERR_INVALID for another mode. */
#define PA_BATCH_FUSED 0
#define PA_BATCH_STREAMS 1
int pa_batch_set_mode(pa_batch* batch, int32_t mode);
/* Kernels launched by pa_batch_run so far (each graph launch counts the kernels it
 * holds) and CUDA graph launches. */
int pa_batch_launches(const pa_batch* batch, int64_t* kernel_launches, int64_t* graph_launches);
/* Borrowed view of run i (valid until pa_batch_destroy), for observables. */
int pa_batch_ctx(pa_batch* batch, int32_t i, pa_ctx** view);
int pa_batch_destroy(pa_batch* batch);

/* Continuous-batching server: submitted runs wait in a FIFO queue and are
 * admitted while the sum of admitted footprints stays within mem_budget bytes
 * and at most max_active runs are on the GPU; every pa_server_poll issues up to
 * steps_per_poll steps of each admitted run, retires runs whose last step has
 * completed on the device (freeing their memory), admits waiting runs, and
 * reports the ids that finished.  A run's stream priority follows its work
 * (Metropolis updates of its schedule), one level per decade, smaller runs
 * higher: the device runs short requests first and fills the rest with long
 * ones. */
typedef struct pa_server pa_server;
int pa_server_create(size_t mem_budget, int32_t max_active, int32_t steps_per_poll, pa_server** out);
int pa_server_submit(pa_server* server, const pa_config* cfg, uint64_t* request_id);
int pa_server_poll(pa_server* server, uint64_t* done_ids, int32_t cap, int32_t* n_done);
/* Observables of population pop at the last step of a finished request with +-1
 * couplings (pa_server_result) or Gaussian couplings (pa_server_gresult), and
 * that step's index; PA_ERR_STATE if the request has not finished, PA_ERR_INVALID
 * for a population it does not have or the other model's reader, the request's
 * own error status if it failed. */
int pa_server_result(pa_server* server, uint64_t request_id, int32_t pop, pa_obs* out, int32_t* last_step);
int pa_server_gresult(pa_server* server, uint64_t request_id, int32_t pop, pa_gobs* out, int32_t* last_step);
/* Requests waiting and running. */
int pa_server_load(pa_server* server, int32_t* queued, int32_t* active);
int pa_server_destroy(pa_server* server);

/* ---- checkpoint and restore ----
 * The state between two steps is device data only (the random streams are
 * counter-based, so there is no generator state): the current population
 * (spins, labels, levels), the step records, level and overlap histograms of
 * steps 0..t, the last copy numbers and parent map, the family-size histogram,
 * and the schedule so far; for Gaussian couplings the energies (int64 fixed
 * point) and Gaussian step records replace levels and level histograms, and the
 * link-overlap histograms are kept too.  A run restored from a checkpoint continues exactly
 * as the original would have.  The paper has no counterpart (its runs are
 * single CPU jobs); long runs at large R need it.
 *
 * pa_checkpoint synchronises, sets *size to the checkpoint's length and, if buf
 * holds at least that many bytes (host memory), writes it; otherwise it returns
 * PA_ERR_CAPACITY and writes nothing (call with buf = NULL to size a buffer).
 * The format is this library's, in host byte order, not a portable archive. */
int pa_checkpoint(pa_ctx* ctx, void* buf, size_t cap, size_t* size);

/* Creates a run on cuda_stream from a checkpoint of a run with the same
 * configuration (same model, sizes, seeds, schedule or adaptive target; a
 * different configuration or a damaged buffer gives PA_ERR_INVALID).  The new context
 * owns its memory like one from pa_create. */
int pa_restore(const pa_config* cfg, const void* buf, size_t size, void* cuda_stream, pa_ctx** out);

/* ---- launch shapes of the sweep kernel and their autotuner ----
 * An implementation choice with no counterpart in the paper.  The sweep kernel
 * (+-1 couplings) is compiled for a few launch shapes per lattice size L: W
 * words per site row (a CTA holds 32W replicas, one bit each, all N sites, in
 * shared memory), threads per CTA,
 * and the CTAs per SM it is compiled for.  Every shape gives bit-identical
 * results (the random words depend on slot and site, never on the tiling); they
 * differ only in speed.  The first shape of each L is the default.  A run uses
 * the shape selected for its L on the current device when it is created; when
 * that choice is the default or the autotuner's (not pinned by pa_sweep_select
 * with an index) and the run's population gives fewer tiles than the device has
 * SMs, it takes the shape of that L with the most tiles instead. */
typedef struct {
  int32_t L;
  int32_t words;         /* W: 32-bit words per site row of a tile (32 replicas each) */
  int32_t threads;       /* threads per CTA */
  int32_t ctas_per_sm;   /* CTAs per SM the kernel is compiled for (register cap) */
  int32_t smem_bytes;    /* dynamic shared memory per CTA */
} pa_sweep_shape;

/* The shapes compiled for L, default first: *n = their number; up to cap are
 * written to shapes (which may be NULL when cap is 0).  No GPU is needed. */
int pa_sweep_shapes(int32_t L, pa_sweep_shape* shapes, int32_t cap, int32_t* n);

/* Selects shape `index` of L for runs created afterwards on the current
 * device (-1: the default).  Thread-safe. */
int pa_sweep_select(int32_t L, int32_t index);
int pa_sweep_selected(int32_t L, int32_t* index);

/* The sweep launches of run c: *shape = the index (into pa_sweep_shapes(L)) of the
 * shape its tiles use; when the population leaves the last wave of tiles mostly
 * empty (the run's R replicas fill at least one wave of the device's SMs and a
 * last wave at most 60 % full), that wave is a second launch of the next smaller
 * tile shape: *tail_shape = its index and *tail_from = the first slot it covers
 * (a multiple of both tile sizes); otherwise *tail_shape = -1 and *tail_from = 0.
 * Both launches give the results of one.  Runs of the Gaussian model, sharded
 * runs and runs whose shape is pinned with pa_sweep_select have no second launch.
 * PA_ERR_INVALID for a NULL argument. */
int pa_sweep_plan(const pa_ctx* c, int32_t* shape, int32_t* tail_shape, int32_t* tail_from);

/* Autotuner: on the current device, creates a scratch run of size L with R
 * replicas (one population, one temperature step from beta 0 to 0.5, 10
 * sweeps), times `launches` sweep launches of every shape of L (after one
 * untimed launch each) with CUDA events, selects the fastest for L and returns
 * its index in *best.  ms_per_launch, if not NULL, receives up to cap per-shape
 * times (a shape that cannot launch on this device gets a negative time).  The
 * scratch run's memory is freed before returning; PA_ERR_NOMEM if it does not
 * fit. */
int pa_sweep_autotune(int32_t L, int32_t R, int32_t launches, double* ms_per_launch, int32_t cap, int32_t* best);

/* ---- resampling without device allocation ----
 * The paper has no counterpart: this is a service entry point for callers that
 * cannot allocate device memory — code that runs under a framework's allocator
 * that owns all device memory (a raw cudaMalloc there fails or fragments the
 * pool), latency-critical loops in which cudaMalloc/cudaFree would synchronise
 * the device, and deployments that budget device memory exactly.
 *
 * It computes what pa_step's resampling computes, on caller-owned DEVICE
 * buffers: for old slots i < n_old with energy level levels[i] (unsatisfied
 * bonds), the copy numbers counts[i] = fl[k] + [r_i < thr[k]] with
 * r_i = word (i & 3) of Philox4x32-10 keyed by (run_seed, resampling, pop) at
 * counter (i >> 2, 0, 0, t): floor(tau) copies, plus one more when the uniform
 * word falls below the fraction of tau scaled to 2^32; the parent of every new
 * slot j < min(*n_new, parents_cap) (parents[j] = i for
 * offset_i <= j < offset_i + n_i, offsets the exclusive scan of the counts);
 * and *n_new = sum_i n_i (device int64, exact up to 2^63; parents beyond
 * parents_cap are not written, so the caller compares *n_new with
 * parents_cap).  fl and thr hold n_levels entries (floor(tau_k) and
 * 2^32 frac(tau_k), as pa_step uses them).
 *
 * Invalid device data is reported on the device, not clamped: when a level lies
 * outside [0, n_levels) or an fl entry outside [0, 2^31 - 2], the slot's count
 * is written as 0, *n_new is set to -1 and no parent is written.  Nothing is
 * ever written outside counts[0, n_old) and parents[0, parents_cap).
 *
 * It allocates nothing: its scratch (the per-block totals and offsets of the
 * scan and an error mark) is a fixed array of 4097 64-bit words (about 32 KiB)
 * in the library's device memory, held by every GPU that loads the library
 * until the process exits, which limits n_old to PA_NOALLOC_MAX_SLOTS (larger
 * inputs return PA_ERR_INVALID before any launch).  All calls on a device share
 * that array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The first call on a
 * device looks up the array's device address (once per device, with that device
 * current), so make that first call before any stream capture.  The address is
 * kept for the life of the process: do not call this entry point on a device
 * after cudaDeviceReset (or any other teardown of its primary context) in the
 * same process.  Asynchronous on `cuda_stream` (NULL = legacy default stream);
 * returns PA_OK, PA_ERR_INVALID or PA_ERR_CUDA. */
#define PA_NOALLOC_MAX_BLOCKS 4096
#define PA_NOALLOC_MAX_SLOTS (PA_NOALLOC_MAX_BLOCKS * 1024)
int pa_resample_counts_noalloc(const int32_t* levels, int64_t n_old, const int32_t* fl, const uint32_t* thr,
                               int32_t n_levels, uint64_t run_seed, int32_t pop, int32_t t, int32_t* counts,
                               int32_t* parents, int64_t parents_cap, int64_t* n_new, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PA_H */
