/* pa_oracle.h — plain, slow CPU oracle for population annealing (PA) on the
 * 3D Edwards-Anderson spin glass with +-1 couplings.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library: every step here is written from the paper (Amey & Machta,
 * "Analysis and Optimization of Population Annealing", §II and §III.C).
 *
 * Conventions (the paper is silent on them; the readings are listed in the
 * design notes):
 *   - sites n = x + L*(y + L*z); bond (n,d) joins n and n+e_d (periodic),
 *     d = 0:x, 1:y, 2:z, so a lattice has 3N bonds (at L=2 two distinct bonds
 *     join each neighbouring pair);
 *   - energy E = -sum_n sum_d J(n,d) s_n s_{n+e_d}; level k = (E + 3N)/2 is
 *     the number of unsatisfied bonds, 0 <= k <= 3N;
 *   - temperature index t ascends from beta_0 = 0 (the paper's index runs
 *     the other way);
 *   - random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *     (seed, purpose, population) and countered by (site, sweep, slot, step).
 */
#ifndef PA_ORACLE_H
#define PA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_P_COUPLINGS = 0, OR_P_INIT = 1, OR_P_METROPOLIS = 2, OR_P_RESAMPLE = 3 };

enum { OR_OK = 0, OR_DONE = 1, OR_ERR_INVALID = -1, OR_ERR_NOMEM = -2, OR_ERR_CAPACITY = -3 };

typedef struct {
  int32_t L;                      /* even L >= 2, or L = 3 (three-colour sweep) */
  int64_t R;                      /* target population size */
  int64_t R_cap;                  /* hard capacity of the population arrays */
  uint64_t disorder_seed;         /* couplings, < 2^56 */
  uint64_t run_seed;              /* spins, Metropolis and resampling, < 2^56 */
  int32_t n_pop;                  /* 1, or 2 independent populations on one disorder */
  int32_t n_temps;                /* explicit schedule length, or the step limit when adaptive */
  const double* betas;            /* ascending, betas[0] = 0; NULL => adaptive schedule */
  double beta_max;                /* adaptive only: last inverse temperature */
  double eps_target;              /* adaptive only: culling fraction to hold */
  int32_t n_sweeps;               /* sweeps per step when sweeps_per_step is NULL */
  const int32_t* sweeps_per_step; /* per-step sweep counts (index t), or NULL */
  int32_t q_bins;                 /* overlap histogram bins (odd, >= 3) */
  int32_t n_threads;              /* OpenMP threads, 0 = runtime default */
} or_config;

/* Per-step, per-population record (all values refer to step t, measured after
 * the sweeps at beta_t; the resampling fields describe the move beta_{t-1} -> beta_t). */
typedef struct {
  int32_t t;
  double beta, dbeta;
  int64_t R_tilde;          /* population size at step t */
  int64_t sum_E, sum_E2;    /* exact integer sums over the population */
  int32_t E_min;            /* lowest energy in the population at t */
  double mean_E, var_E;
  int32_t kmin_prev;        /* lowest level of the step t-1 population */
  double S_prime;           /* sum_k c_{t-1}(k) exp(-dbeta*2*(k-kmin)) */
  double lnQ;               /* ln Q(beta_{t-1}, beta_t), Eq. (Q) */
  double minus_beta_F;      /* -beta_t F~(beta_t), Eq. (betaF) */
  double eps_expected;      /* Eq. (eq_num_elim) divided by R */
  int64_t culled;           /* replicas that received zero copies */
  int64_t sum_eta2;         /* sum over families of eta^2 */
  int64_t n_families;       /* families with at least one member */
  double rho_t;             /* sum eta^2 / R_tilde */
  double S_f;               /* family entropy -sum nu ln nu, nu = eta/R_tilde */
  double rho_s;             /* R_tilde / exp(S_f) */
  int32_t E0;               /* lowest energy measured up to and including t */
  double g0_tilde;          /* fraction of the population at E0 */
  double g0_bar;            /* 2 exp(-beta E0 + beta F~), Eq. (g0) */
  int64_t q_pairs;          /* overlap pairs (two populations only) */
  int64_t q_abs_le_02;      /* pairs with |q| <= 0.2 */
  double I02;               /* q_abs_le_02 / q_pairs */
} or_obs;

typedef struct or_run or_run;

/* ---- building blocks (exported so tests can pin them one by one) ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_key(uint64_t seed, uint32_t purpose, uint32_t pop, uint32_t key[2]);
/* J[3*n + d] = +1/-1 from the disorder seed */
void or_couplings(int32_t L, uint64_t disorder_seed, int8_t* J);
int32_t or_energy(int32_t L, const int8_t* J, const int8_t* s);
/* Metropolis thresholds for dE = 4, 8, 12 at inverse temperature beta */
void or_metropolis_thresholds(double beta, uint32_t thr[3]);
/* The 32-bit Metropolis uniform of replica `slot` at one site and half-sweep (its
 * bit column across the stream's words), and the test uniform < thr read from the
 * top bit down, stopping at the first bit where the two differ */
uint32_t or_metropolis_uniform(uint64_t run_seed, int32_t pop, uint32_t site_index, uint32_t half_sweep,
                               int64_t slot, int32_t t);
int32_t or_metropolis_test(uint64_t run_seed, int32_t pop, uint32_t site_index, uint32_t half_sweep, int64_t slot,
                           int32_t t, uint32_t thr);
/* S sweeps of one replica (slot j) at step t, in place; returns the energy change */
int32_t or_sweep_replica(int32_t L, const int8_t* J, int8_t* s, uint64_t run_seed, int32_t pop,
                         int64_t slot, int32_t t, int32_t n_sweeps, const uint32_t thr[3]);
/* Reweighting of a level histogram c[0..3N] from one step to the next (Eqs. tau, Q,
 * eq_num_elim).  Writes floor(tau_k) and the 32-bit fraction threshold for every
 * level k >= kmin; returns kmin, or -1 for an empty histogram. */
int32_t or_reweight(int32_t n_levels, const int64_t* c, int64_t R, double dbeta, double* S_prime,
                    int32_t* fl, uint32_t* thr, double* eps_expected);
/* Copies of one replica at old slot i under the nearest-integer rule */
int32_t or_copy_count(uint64_t run_seed, int32_t pop, int32_t t, int64_t i, int32_t fl, uint32_t thr);
/* Nearest-integer resampling of arbitrary expected copy numbers tau[0..n) (used to
 * check the resampling law and the family process on synthetic weights). */
void or_copy_counts(uint64_t run_seed, int32_t pop, int32_t t, int64_t n, const int32_t* levels, const int32_t* fl,
                    const uint32_t* thr, int32_t* out);
void or_resample_uniforms(uint64_t run_seed, int32_t pop, int32_t t, int64_t n, uint32_t* r);
void or_resample_tau(int64_t n, const double* tau, uint64_t seed, int32_t pop, int32_t t, int32_t* n_out);
/* Exact density of states g[k], k = 0..3N, by enumerating all 2^N states (N <= 30) */
int or_enumerate_levels(int32_t L, const int8_t* J, int64_t* g);

/* ---- full runs ---- */
int or_create(const or_config* cfg, or_run** out);
int or_step(or_run* run);             /* OR_OK, OR_DONE after the last step, or an error */
int or_run_all(or_run* run);
int32_t or_current_step(const or_run* run);
int or_observables(const or_run* run, int32_t t, int32_t pop, or_obs* out);
/* energy-level histogram c_t(k) of population pop at step t (3N+1 entries) */
int or_energy_hist(const or_run* run, int32_t t, int32_t pop, int64_t* out);
/* family-size histogram at the current step: eta[i], m[i] for i < *n (ascending eta) */
int or_family_hist(const or_run* run, int32_t pop, int64_t cap, int64_t* eta, int64_t* m, int64_t* n);
/* overlap histogram at step t (q_bins entries) */
int or_q_hist(const or_run* run, int32_t t, int64_t* out);
/* current population: spins [count][N] replica-major, labels, energies */
int or_population(const or_run* run, int32_t pop, int64_t cap, int8_t* spins, int32_t* labels,
                  int32_t* energies, int64_t* count);
/* copy numbers n_i of the last resampling (old slots), and the old population size */
int or_last_counts(const or_run* run, int32_t pop, int64_t cap, int32_t* counts, int64_t* count);
const int8_t* or_couplings_of(const or_run* run);
double or_beta(const or_run* run, int32_t t);
void or_destroy(or_run* run);

/* ---- Gaussian couplings (the paper's model, §II.A): pa_oracle_gauss.c ----
 * Couplings J ~ N(0,1) clamped to [-5, 5] in fixed point Jq = round(J 2^20);
 * energies in the same units (int64).  Explicit or adaptive schedules, even L. */

typedef struct {
  int32_t t;
  double beta, dbeta;
  int64_t R_tilde;
  int64_t sum_E;            /* exact, units of 2^-20 */
  double sum_E2;            /* exact 128-bit sum of E^2 rounded to double, units of 2^-40 */
  int64_t E_min;            /* lowest energy at t */
  double mean_E, var_E;     /* in units of J */
  int64_t E_min_prev;       /* lowest energy of the step t-1 population */
  double S_prime, lnQ, minus_beta_F, eps_expected;
  int64_t culled, sum_eta2, n_families;
  double rho_t, S_f, rho_s;
  int64_t E0;               /* lowest energy measured up to t */
  double g0_tilde, g0_bar;
  int64_t q_pairs, q_abs_le_02;
  double I02;
  int64_t ql_sum;           /* sum over pairs of sum over bonds s1 s1 s2 s2 */
  double ql_mean;           /* <q_l>, Eq. (ql) */
  double e_l;               /* Eq. (el) */
  double delta_KY;          /* e_l - <E>/N for this disorder sample (Eq. KY before the disorder average) */
} org_obs;

typedef struct org_run org_run;

void org_couplings(int32_t L, uint64_t disorder_seed, int32_t* Jq);
int64_t org_energy(int32_t L, const int32_t* Jq, const int8_t* s);
/* Metropolis threshold of a flip costing dE > 0 (fixed point, units of 2^-20) */
uint32_t org_acceptance_threshold(double beta, int64_t dE);
/* The 32-bit uniform of replica `slot` at site n in half-sweep (sweep, colour) of
 * step t: upper 16 bits from half (slot & 1) of word (slot >> 1) & 3 of Philox at
 * counter (n >> 1, 2 sweep + colour, slot >> 3, t), lower 16 bits from the upper half
 * of word slot & 3 at counter (n >> 1, 2 sweep + colour, (slot >> 2) | 2^31, t). */
uint32_t org_metropolis_uniform(uint64_t run_seed, int32_t pop, int32_t n, int32_t sweep, int32_t colour,
                                int64_t slot, int32_t t);
int64_t org_sweep_replica(int32_t L, const int32_t* Jq, int8_t* s, uint64_t run_seed, int32_t pop, int64_t slot,
                          int32_t t, int32_t n_sweeps, double beta);
/* resampling weight exp(-dbeta d 2^-20) of a replica d above the lowest energy */
double org_weight(double dbeta, int64_t d);
/* E_min, S' = sum_i w_i, (1/R) sum_{tau_i<1} (1 - tau_i), and tau_i (if tau != NULL) */
int org_reweight(const int64_t* E, int64_t n, int64_t R, double dbeta, int64_t* E_min, double* S_prime,
                 double* eps_expected, double* tau);
int org_create(const or_config* cfg, org_run** out);
int org_step(org_run* run);
int org_run_all(org_run* run);
int32_t org_current_step(const org_run* run);
int org_observables(const org_run* run, int32_t t, int32_t pop, org_obs* out);
int org_q_hist(const org_run* run, int32_t t, int32_t link, int64_t* out);
int org_population(const org_run* run, int32_t pop, int64_t cap, int8_t* spins, int32_t* labels, int64_t* E,
                   int64_t* n);
int org_last_counts(const org_run* run, int32_t pop, int64_t cap, int32_t* counts, int64_t* n);
const int32_t* org_couplings_of(const org_run* run);
void org_destroy(org_run* run);

#ifdef __cplusplus
}
#endif
#endif
