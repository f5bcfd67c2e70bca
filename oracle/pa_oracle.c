/* pa_oracle.c — plain, slow CPU oracle for population annealing (PA).
 *
 * TEST INFRASTRUCTURE ONLY: this file is the reference the CUDA path is checked
 * against.  It is written for a reader holding the paper (Amey & Machta,
 * "Analysis and Optimization of Population Annealing"), step by step in the
 * paper's order, with no blocking, fusion or reordering.  It shares nothing
 * with the CUDA library.  Build with -ffp-contract=off so that every floating
 * point expression below rounds exactly as written.
 *
 * Parity status of each function (what pins it is in tests/):
 *   or_philox4x32_10     pinned: independent Philox implementation, many counters/keys
 *   or_couplings         pinned: +-1 balance, determinism
 *   or_energy            pinned: ferromagnet / Neel ground states, enumeration identities
 *   or_enumerate_levels  pinned: sum g = 2^N, g(E) = g(-E) for even L, beta=0 variance 3N,
 *                        ferromagnet degeneracies, gauge invariance, high-T expansion
 *   or_metropolis_uniform pinned: the bit-column uniform is uniform and independent
 *                        between slots, half-sweeps and populations
 *   or_metropolis_test   pinned: equals the plain comparison of the full bit-column uniform
 *   or_sweep_replica     pinned: Boltzmann energy distribution vs enumeration (L=2, 3)
 *   or_reweight          pinned: sum_k c_k tau_k = R, tau ratios = Boltzmann ratios
 *   or_copy_count / or_resample_tau
 *                        pinned: E[n] = tau, var n = f(1-f), eps = E(1-tau)_+,
 *                        sum var z = 2 eps - 2 pi eps^2 (Appendix B), family law Eq. (petak)
 *   full run             pinned: -beta F~ vs exact ln Z, <E> vs exact, E0 vs exact ground
 *                        state, culled fraction vs Eq. (eq_num_elim), overlap vs exact P(q)
 */
#include "pa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11).  Each round multiplies counter words 0 and 2 by the two
 * round multipliers, and mixes the high halves with the other two words and the
 * key; the key is bumped by the two Weyl constants between rounds. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Key of one random stream: seed (< 2^56) plus a 4-bit purpose and a 4-bit
 * population index packed above it. */
void or_key(uint64_t seed, uint32_t purpose, uint32_t pop, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32) | (purpose << 28) | (pop << 24);
}

static uint32_t philox_word(const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                            int which) {
  uint32_t ctr[4] = {c0, c1, c2, c3}, out[4];
  or_philox4x32_10(ctr, key, out);
  return out[which];
}

/* ------------------------------------------------------------------------- */
/* Lattice and Hamiltonian, §II.A: H = -sum_<nm> J_nm s_n s_m on a periodic
 * cubic lattice.  The paper draws J from a Gaussian; this oracle follows the
 * +-1 (bimodal) couplings of the workloads it checks. */

static int32_t site(int32_t L, int32_t x, int32_t y, int32_t z) {
  x = (x % L + L) % L;
  y = (y % L + L) % L;
  z = (z % L + L) % L;
  return x + L * (y + L * z);
}

static int32_t neighbour(int32_t L, int32_t n, int32_t d, int32_t dir) {
  int32_t x = n % L, y = (n / L) % L, z = n / (L * L);
  if (d == 0) x += dir;
  if (d == 1) y += dir;
  if (d == 2) z += dir;
  return site(L, x, y, z);
}

void or_couplings(int32_t L, uint64_t disorder_seed, int8_t* J) {
  int32_t N = L * L * L;
  uint32_t key[2];
  or_key(disorder_seed, OR_P_COUPLINGS, 0, key);
  for (int32_t n = 0; n < N; ++n) {
    for (int32_t d = 0; d < 3; ++d) {
      uint32_t r = philox_word(key, (uint32_t)n, 0, 0, 0, d);
      J[3 * n + d] = (r & 1u) == 0 ? 1 : -1;
    }
  }
}

int32_t or_energy(int32_t L, const int8_t* J, const int8_t* s) {
  int32_t N = L * L * L;
  int32_t E = 0;
  for (int32_t n = 0; n < N; ++n)
    for (int32_t d = 0; d < 3; ++d) E -= J[3 * n + d] * s[n] * s[neighbour(L, n, d, +1)];
  return E;
}

/* Local field h_n = sum over the six bonds touching n of J * s_neighbour. */
static int32_t local_field(int32_t L, const int8_t* J, const int8_t* s, int32_t n) {
  int32_t h = 0;
  for (int32_t d = 0; d < 3; ++d) {
    int32_t up = neighbour(L, n, d, +1);
    int32_t dn = neighbour(L, n, d, -1);
    h += J[3 * n + d] * s[up];
    h += J[3 * dn + d] * s[dn];
  }
  return h;
}

/* ------------------------------------------------------------------------- */
/* Metropolis MCMC at fixed beta (§II: "an MCMC procedure such as the Metropolis
 * algorithm").  dE <= 0 is always accepted; a flip costing dE > 0 is accepted when
 * the replica's 32-bit uniform r is below thr = floor(2^32 exp(-beta dE)).
 *
 * r is the replica's bit column in the Metropolis stream: bit 31 - p of r
 * (p = 0 .. 31) is bit (slot mod 32) of word (p mod 4) of the Philox block at
 * counter (site, half-sweep, 8 floor(slot / 32) + floor(p / 4), t).  The sweep
 * below draws the whole uniform and compares it with thr.  or_metropolis_test is
 * the same comparison read from the top bit down, stopping at the first bit where
 * r and thr differ (r < thr exactly when there r has 0 and thr has 1); it is kept
 * as a separate helper, pinned against the plain comparison, because the CUDA
 * path decides its flips that way. */

void or_metropolis_thresholds(double beta, uint32_t thr[3]) {
  for (int m = 1; m <= 3; ++m) {
    double p = exp(-(beta * (double)(4 * m)));
    double v = floor(ldexp(p, 32));
    if (v > 4294967295.0) v = 4294967295.0;
    thr[m - 1] = (uint32_t)v;
  }
}

static void metropolis_block(const uint32_t key[2], uint32_t site_index, uint32_t half_sweep, int64_t slot, int p,
                             int32_t t, uint32_t out[4]) {
  uint32_t ctr[4] = {site_index, half_sweep, (uint32_t)(8 * (slot >> 5) + (p >> 2)), (uint32_t)t};
  or_philox4x32_10(ctr, key, out);
}

uint32_t or_metropolis_uniform(uint64_t run_seed, int32_t pop, uint32_t site_index, uint32_t half_sweep,
                               int64_t slot, int32_t t) {
  uint32_t key[2], out[4], r = 0;
  or_key(run_seed, OR_P_METROPOLIS, (uint32_t)pop, key);
  for (int p = 0; p < 32; ++p) {
    if ((p & 3) == 0) metropolis_block(key, site_index, half_sweep, slot, p, t, out);
    r |= ((out[p & 3] >> (slot & 31)) & 1u) << (31 - p);
  }
  return r;
}

static int32_t test_below(const uint32_t key[2], uint32_t site_index, uint32_t half_sweep, int64_t slot, int32_t t,
                          uint32_t thr) {
  uint32_t out[4];
  for (int p = 0; p < 32; ++p) {
    if ((p & 3) == 0) metropolis_block(key, site_index, half_sweep, slot, p, t, out);
    uint32_t r_bit = (out[p & 3] >> (slot & 31)) & 1u, thr_bit = (thr >> (31 - p)) & 1u;
    if (r_bit != thr_bit) return r_bit < thr_bit;
  }
  return 0; /* r == thr */
}

int32_t or_metropolis_test(uint64_t run_seed, int32_t pop, uint32_t site_index, uint32_t half_sweep, int64_t slot,
                           int32_t t, uint32_t thr) {
  uint32_t key[2];
  or_key(run_seed, OR_P_METROPOLIS, (uint32_t)pop, key);
  return test_below(key, site_index, half_sweep, slot, t, thr);
}

static int32_t n_colours(int32_t L) { return (L % 2 == 0) ? 2 : 3; }

int32_t or_sweep_replica(int32_t L, const int8_t* J, int8_t* s, uint64_t run_seed, int32_t pop,
                         int64_t slot, int32_t t, int32_t n_sweeps, const uint32_t thr[3]) {
  int32_t ncol = n_colours(L);
  int32_t dE_total = 0;
  for (int32_t sw = 0; sw < n_sweeps; ++sw) {
    for (int32_t c = 0; c < ncol; ++c) {
      for (int32_t z = 0; z < L; ++z)
        for (int32_t y = 0; y < L; ++y)
          for (int32_t x = 0; x < L; ++x) {
            if ((x + y + z) % ncol != c) continue;
            int32_t n = site(L, x, y, z);
            int32_t h = local_field(L, J, s, n);
            int32_t dE = 2 * s[n] * h;
            uint32_t site_index = (ncol == 2) ? (uint32_t)(n >> 1) : (uint32_t)n;
            uint32_t half_sweep = (uint32_t)(ncol * sw + c);
            if (dE <= 0 || or_metropolis_uniform(run_seed, pop, site_index, half_sweep, slot, t) < thr[dE / 4 - 1]) {
              s[n] = (int8_t)(-s[n]);
              dE_total += dE;
            }
          }
    }
  }
  return dE_total;
}

/* ------------------------------------------------------------------------- */
/* Resampling, §II, Eqs. (tau) and (Q).  Replicas with equal energy have equal
 * weights, so the sum of Eq. (Q) is taken level by level, ascending, with every
 * weight measured from the lowest level present (E_min) to keep it <= 1:
 *   S' = sum_k c(k) exp(-dbeta (E_k - E_min)),  E_k - E_min = 2 (k - kmin)
 *   tau_k = (R / R~) e^{-dbeta E_k} / Q = R exp(-dbeta (E_k - E_min)) / S'.
 * The expected culling fraction is Eq. (eq_num_elim) divided by R. */

int32_t or_reweight(int32_t n_levels, const int64_t* c, int64_t R, double dbeta, double* S_prime,
                    int32_t* fl, uint32_t* thr, double* eps_expected) {
  int32_t kmin = -1;
  for (int32_t k = 0; k < n_levels; ++k)
    if (c[k] > 0) {
      kmin = k;
      break;
    }
  if (kmin < 0) return -1;
  double S = 0.0;
  for (int32_t k = kmin; k < n_levels; ++k) {
    double w = exp(-(dbeta * (double)(2 * (k - kmin))));
    S = S + (double)c[k] * w;
  }
  double eps = 0.0;
  for (int32_t k = kmin; k < n_levels; ++k) {
    double w = exp(-(dbeta * (double)(2 * (k - kmin))));
    double tau = ((double)R * w) / S;
    double f = floor(tau);
    if (fl) fl[k] = (int32_t)f;
    if (thr) thr[k] = (uint32_t)((tau - f) * 4294967296.0);
    if (tau < 1.0) eps = eps + (double)c[k] * (1.0 - tau);
  }
  *S_prime = S;
  *eps_expected = eps / (double)R;
  return kmin;
}

/* Nearest-integer resampling (§II): floor(tau) copies with probability
 * ceil(tau) - tau, else ceil(tau).  The uniform word r is compared with the
 * fraction of tau scaled to 2^32. */
int32_t or_copy_count(uint64_t run_seed, int32_t pop, int32_t t, int64_t i, int32_t fl, uint32_t thr) {
  uint32_t key[2];
  or_key(run_seed, OR_P_RESAMPLE, (uint32_t)pop, key);
  uint32_t r = philox_word(key, (uint32_t)(i >> 2), 0, 0, (uint32_t)t, (int)(i & 3));
  return fl + (r < thr ? 1 : 0);
}

/* Copy numbers of old slots 0..n-1 whose energy levels are given, from per-level
 * tables of floor(tau) and 2^32 frac(tau) (the rule above, tau taken per level). */
void or_copy_counts(uint64_t run_seed, int32_t pop, int32_t t, int64_t n, const int32_t* levels, const int32_t* fl,
                    const uint32_t* thr, int32_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = or_copy_count(run_seed, pop, t, i, fl[levels[i]], thr[levels[i]]);
}

/* The uniform words r_i that the resampling at step t draws for old slots 0..n-1. */
void or_resample_uniforms(uint64_t run_seed, int32_t pop, int32_t t, int64_t n, uint32_t* r) {
  uint32_t key[2];
  or_key(run_seed, OR_P_RESAMPLE, (uint32_t)pop, key);
  for (int64_t i = 0; i < n; ++i) r[i] = philox_word(key, (uint32_t)(i >> 2), 0, 0, (uint32_t)t, (int)(i & 3));
}

void or_resample_tau(int64_t n, const double* tau, uint64_t seed, int32_t pop, int32_t t, int32_t* n_out) {
  for (int64_t i = 0; i < n; ++i) {
    double f = floor(tau[i]);
    uint32_t thr = (uint32_t)((tau[i] - f) * 4294967296.0);
    n_out[i] = or_copy_count(seed, pop, t, i, (int32_t)f, thr);
  }
}

/* ------------------------------------------------------------------------- */
/* Exact enumeration of all 2^N states in Gray-code order: consecutive states
 * differ in one spin, whose flip changes E by 2 s_n h_n.  E(s) = E(-s), so only
 * the half with the last spin up is visited and every count is doubled.  The
 * six (neighbour, coupling) pairs of each site are tabulated once. */
int or_enumerate_levels(int32_t L, const int8_t* J, int64_t* g) {
  int32_t N = L * L * L;
  if (N > 30) return OR_ERR_INVALID;
  int8_t s[32];
  int32_t nb[32][6];
  int32_t jb[32][6];
  for (int32_t n = 0; n < N; ++n) {
    s[n] = 1;
    for (int32_t d = 0; d < 3; ++d) {
      int32_t up = neighbour(L, n, d, +1);
      int32_t dn = neighbour(L, n, d, -1);
      nb[n][2 * d] = up;
      jb[n][2 * d] = J[3 * n + d];
      nb[n][2 * d + 1] = dn;
      jb[n][2 * d + 1] = J[3 * dn + d];
    }
  }
  memset(g, 0, sizeof(int64_t) * (size_t)(3 * N + 1));
  int32_t E = or_energy(L, J, s);
  g[(E + 3 * N) / 2] += 2;
  uint64_t total = (uint64_t)1 << (N - 1);
  for (uint64_t i = 1; i < total; ++i) {
    int32_t n = __builtin_ctzll(i); /* the bit that changes between Gray codes i-1 and i */
    int32_t h = 0;
    for (int b = 0; b < 6; ++b) h += jb[n][b] * s[nb[n][b]];
    E += 2 * s[n] * h;
    s[n] = (int8_t)(-s[n]);
    g[(E + 3 * N) / 2] += 2;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* The population annealing run, §II: a population starts at beta = 0 and is
 * cooled step by step; each step resamples beta_{t-1} -> beta_t, then runs
 * S_t Metropolis sweeps at beta_t, then measures. */

typedef struct {
  int8_t* s[2];      /* double-buffered spins, [slot][site] */
  int32_t* lab[2];   /* family labels */
  int32_t* E[2];     /* energies */
  int cur;
  int64_t Rt;        /* current population size */
  int32_t* counts;   /* copy numbers of the last resampling */
  int64_t counts_n;
  int32_t E0;        /* lowest energy measured so far */
  double lnQ_sum;
} or_pop;

struct or_run {
  or_config cfg;
  int32_t L, N, n_levels, ncol;
  int8_t* J;
  double* betas;     /* [n_temps] */
  int32_t* sweeps;   /* [n_temps] */
  int32_t t;         /* index of the last completed step */
  int done;
  or_pop pops[2];
  or_obs* obs;       /* [n_temps][n_pop] */
  int64_t* hist;     /* [n_temps][n_pop][n_levels] */
  int64_t* qhist;    /* [n_temps][q_bins] */
};

static or_obs* obs_at(const or_run* r, int32_t t, int32_t p) { return &r->obs[(size_t)t * r->cfg.n_pop + p]; }
static int64_t* hist_at(const or_run* r, int32_t t, int32_t p) {
  return &r->hist[((size_t)t * r->cfg.n_pop + p) * r->n_levels];
}

static void set_threads(const or_run* r) {
#ifdef _OPENMP
  if (r->cfg.n_threads > 0) omp_set_num_threads(r->cfg.n_threads);
#else
  (void)r;
#endif
}

/* Family statistics from the labels, which stay sorted along the slots (they
 * start as the slot index and resampling copies in slot order), §III.A:
 * rho_t = sum_families eta^2 / R~ (Eq. rho_t_def2 with the actual size). */
static int family_stats(const or_pop* P, int64_t* sum_eta2, int64_t* n_fam, double* S_f) {
  const int32_t* lab = P->lab[P->cur];
  int64_t R = P->Rt;
  int64_t s2 = 0, nf = 0;
  double S = 0.0;
  int64_t start = 0;
  for (int64_t j = 1; j <= R; ++j) {
    if (j == R || lab[j] != lab[start]) {
      if (j < R && lab[j] < lab[start]) return OR_ERR_INVALID; /* labels must stay sorted */
      int64_t eta = j - start;
      s2 += eta * eta;
      nf += 1;
      start = j;
    }
  }
  /* family entropy from the size histogram, ascending size */
  int64_t* sizes = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nf > 0 ? nf : 1));
  if (!sizes) return OR_ERR_NOMEM;
  int64_t f = 0;
  start = 0;
  for (int64_t j = 1; j <= R; ++j)
    if (j == R || lab[j] != lab[start]) {
      sizes[f++] = j - start;
      start = j;
    }
  /* counting sort of sizes */
  int64_t maxs = 0;
  for (int64_t i = 0; i < nf; ++i)
    if (sizes[i] > maxs) maxs = sizes[i];
  int64_t* m = (int64_t*)calloc((size_t)maxs + 1, sizeof(int64_t));
  if (!m) {
    free(sizes);
    return OR_ERR_NOMEM;
  }
  for (int64_t i = 0; i < nf; ++i) m[sizes[i]] += 1;
  for (int64_t eta = 1; eta <= maxs; ++eta) {
    if (m[eta] == 0) continue;
    double nu = (double)eta / (double)R;
    S = S - (double)m[eta] * (nu * log(nu));
  }
  free(m);
  free(sizes);
  *sum_eta2 = s2;
  *n_fam = nf;
  *S_f = S;
  return OR_OK;
}

static int measure(or_run* r, int32_t t) {
  int32_t N = r->N;
  for (int32_t p = 0; p < r->cfg.n_pop; ++p) {
    or_pop* P = &r->pops[p];
    int64_t* c = hist_at(r, t, p);
    memset(c, 0, sizeof(int64_t) * (size_t)r->n_levels);
    const int32_t* E = P->E[P->cur];
    int64_t sE = 0, sE2 = 0;
    int32_t Emin = 3 * N + 1;
    for (int64_t j = 0; j < P->Rt; ++j) {
      c[(E[j] + 3 * N) / 2] += 1;
      sE += E[j];
      sE2 += (int64_t)E[j] * E[j];
      if (E[j] < Emin) Emin = E[j];
    }
    or_obs* o = obs_at(r, t, p);
    o->t = t;
    o->beta = r->betas[t];
    o->R_tilde = P->Rt;
    o->sum_E = sE;
    o->sum_E2 = sE2;
    o->E_min = Emin;
    o->mean_E = (double)sE / (double)P->Rt;
    o->var_E = (double)sE2 / (double)P->Rt - o->mean_E * o->mean_E;
    /* Eq. (betaF): -beta_t F~ = sum of ln Q over the steps so far + ln 2^N */
    o->minus_beta_F = (double)N * log(2.0) + P->lnQ_sum;
    if (t == 0 || Emin < P->E0) P->E0 = Emin;
    o->E0 = P->E0;
    o->g0_tilde = (double)c[(P->E0 + 3 * N) / 2] / (double)P->Rt;
    /* Eq. (g0): g0_bar = 2 exp(-beta E0 + beta F~) */
    o->g0_bar = 2.0 * exp(-(o->beta * (double)P->E0) - o->minus_beta_F);
    int rc = family_stats(P, &o->sum_eta2, &o->n_families, &o->S_f);
    if (rc != OR_OK) return rc;
    o->rho_t = (double)o->sum_eta2 / (double)P->Rt;
    o->rho_s = (double)P->Rt / exp(o->S_f);
    o->q_pairs = 0;
    o->q_abs_le_02 = 0;
    o->I02 = 0.0;
  }
  if (r->cfg.n_pop == 2) {
    /* Spin overlap q = (1/N) sum_n s^1_n s^2_n (§II.A) between slot j of the two
     * independent populations. */
    int64_t* qh = &r->qhist[(size_t)t * r->cfg.q_bins];
    memset(qh, 0, sizeof(int64_t) * (size_t)r->cfg.q_bins);
    const or_pop* A = &r->pops[0];
    const or_pop* B = &r->pops[1];
    int64_t pairs = A->Rt < B->Rt ? A->Rt : B->Rt;
    int64_t small = 0;
    int64_t nb = r->cfg.q_bins;
    for (int64_t j = 0; j < pairs; ++j) {
      const int8_t* sa = A->s[A->cur] + (size_t)j * N;
      const int8_t* sb = B->s[B->cur] + (size_t)j * N;
      int64_t Q = 0;
      for (int32_t n = 0; n < N; ++n) Q += sa[n] * sb[n];
      int64_t bin = ((Q + N) * (nb - 1) + N) / (2 * (int64_t)N);
      qh[bin] += 1;
      if (5 * (Q < 0 ? -Q : Q) <= N) small += 1; /* |q| <= 0.2 */
    }
    for (int32_t p = 0; p < 2; ++p) {
      or_obs* o = obs_at(r, t, p);
      o->q_pairs = pairs;
      o->q_abs_le_02 = small;
      o->I02 = pairs > 0 ? (double)small / (double)pairs : 0.0;
    }
  }
  return OR_OK;
}

static void free_run(or_run* r) {
  if (!r) return;
  for (int p = 0; p < 2; ++p) {
    for (int b = 0; b < 2; ++b) {
      free(r->pops[p].s[b]);
      free(r->pops[p].lab[b]);
      free(r->pops[p].E[b]);
    }
    free(r->pops[p].counts);
  }
  free(r->J);
  free(r->betas);
  free(r->sweeps);
  free(r->obs);
  free(r->hist);
  free(r->qhist);
  free(r);
}

int or_create(const or_config* cfg, or_run** out) {
  *out = NULL;
  if (!cfg || cfg->L < 2 || (cfg->L % 2 != 0 && cfg->L != 3) || cfg->R < 1 || cfg->n_temps < 1 ||
      cfg->n_pop < 1 || cfg->n_pop > 2 || cfg->q_bins < 3 || cfg->disorder_seed >= ((uint64_t)1 << 56) ||
      cfg->run_seed >= ((uint64_t)1 << 56) || cfg->R_cap < cfg->R || cfg->R_cap >= ((int64_t)1 << 31))
    return OR_ERR_INVALID;
  if (!cfg->betas && !(cfg->eps_target > 0.0 && cfg->eps_target < 1.0 && cfg->beta_max > 0.0))
    return OR_ERR_INVALID;
  if (cfg->betas) {
    if (cfg->betas[0] != 0.0) return OR_ERR_INVALID;
    for (int32_t t = 1; t < cfg->n_temps; ++t)
      if (!(cfg->betas[t] >= cfg->betas[t - 1])) return OR_ERR_INVALID;
  }
  or_run* r = (or_run*)calloc(1, sizeof(or_run));
  if (!r) return OR_ERR_NOMEM;
  r->cfg = *cfg;
  r->L = cfg->L;
  r->N = cfg->L * cfg->L * cfg->L;
  r->n_levels = 3 * r->N + 1;
  r->ncol = n_colours(cfg->L);
  int32_t N = r->N;
  int32_t T = cfg->n_temps;
  r->J = (int8_t*)malloc((size_t)3 * N);
  r->betas = (double*)calloc((size_t)T, sizeof(double));
  r->sweeps = (int32_t*)calloc((size_t)T, sizeof(int32_t));
  r->obs = (or_obs*)calloc((size_t)T * cfg->n_pop, sizeof(or_obs));
  r->hist = (int64_t*)calloc((size_t)T * cfg->n_pop * r->n_levels, sizeof(int64_t));
  r->qhist = (int64_t*)calloc((size_t)T * cfg->q_bins, sizeof(int64_t));
  if (!r->J || !r->betas || !r->sweeps || !r->obs || !r->hist || !r->qhist) {
    free_run(r);
    return OR_ERR_NOMEM;
  }
  r->cfg.betas = NULL;
  r->cfg.sweeps_per_step = NULL;
  for (int32_t t = 0; t < T; ++t) {
    r->betas[t] = cfg->betas ? cfg->betas[t] : 0.0;
    r->sweeps[t] = cfg->sweeps_per_step ? cfg->sweeps_per_step[t] : cfg->n_sweeps;
  }
  r->cfg.betas = cfg->betas ? r->betas : NULL; /* non-NULL marks an explicit schedule */
  or_couplings(r->L, cfg->disorder_seed, r->J);
  set_threads(r);
  for (int32_t p = 0; p < cfg->n_pop; ++p) {
    or_pop* P = &r->pops[p];
    for (int b = 0; b < 2; ++b) {
      P->s[b] = (int8_t*)malloc((size_t)cfg->R_cap * N);
      P->lab[b] = (int32_t*)malloc(sizeof(int32_t) * (size_t)cfg->R_cap);
      P->E[b] = (int32_t*)malloc(sizeof(int32_t) * (size_t)cfg->R_cap);
      if (!P->s[b] || !P->lab[b] || !P->E[b]) {
        free_run(r);
        return OR_ERR_NOMEM;
      }
    }
    P->counts = (int32_t*)malloc(sizeof(int32_t) * (size_t)cfg->R_cap);
    if (!P->counts) {
      free_run(r);
      return OR_ERR_NOMEM;
    }
    P->cur = 0;
    P->Rt = cfg->R;
    P->lnQ_sum = 0.0;
    uint32_t key[2];
    or_key(cfg->run_seed, OR_P_INIT, (uint32_t)p, key);
    int8_t* s = P->s[0];
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < cfg->R; ++j) {
      for (int32_t n = 0; n < N; ++n) {
        uint32_t w = philox_word(key, (uint32_t)n, 0, (uint32_t)(j >> 2), 0, (int)(j & 3));
        s[(size_t)j * N + n] = (w & 1u) == 0 ? 1 : -1;
      }
      P->lab[0][j] = (int32_t)j;
      P->E[0][j] = or_energy(r->L, r->J, s + (size_t)j * N);
    }
  }
  r->t = 0;
  int rc = measure(r, 0);
  if (rc != OR_OK) {
    free_run(r);
    return rc;
  }
  r->done = (T == 1) || (!cfg->betas && cfg->beta_max <= 0.0);
  *out = r;
  return OR_OK;
}

/* Expected culling fraction of a move by dbeta, for the adaptive schedule. */
static double eps_of(const or_run* r, const int64_t* c, double dbeta) {
  double S, eps;
  or_reweight(r->n_levels, c, r->cfg.R, dbeta, &S, NULL, NULL, &eps);
  return eps;
}

/* Adaptive beta-schedule, §IV.B: hold the culling fraction of Eq. (eq_num_elim)
 * at the target.  The step size is found by bisection on (0, beta_max - beta],
 * 64 halvings, keeping the largest tested step whose culling fraction does not
 * exceed the target; population 0 decides. */
static double choose_dbeta(const or_run* r, int32_t t) {
  double prev = r->betas[t - 1];
  double rem = r->cfg.beta_max - prev;
  const int64_t* c = hist_at(r, t - 1, 0);
  if (eps_of(r, c, rem) <= r->cfg.eps_target) return rem;
  double lo = 0.0, hi = rem;
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi);
    if (eps_of(r, c, mid) <= r->cfg.eps_target)
      lo = mid;
    else
      hi = mid;
  }
  return lo > 0.0 ? lo : hi;
}

int or_step(or_run* r) {
  if (r->done) return OR_DONE;
  int32_t t = r->t + 1;
  int32_t N = r->N;
  double dbeta;
  if (r->cfg.betas) {
    dbeta = r->betas[t] - r->betas[t - 1];
  } else {
    dbeta = choose_dbeta(r, t);
    double b = r->betas[t - 1] + dbeta;
    if (b >= r->cfg.beta_max || dbeta == r->cfg.beta_max - r->betas[t - 1]) b = r->cfg.beta_max;
    r->betas[t] = b;
  }
  uint32_t met[3];
  or_metropolis_thresholds(r->betas[t], met);
  int32_t* fl = (int32_t*)malloc(sizeof(int32_t) * (size_t)r->n_levels);
  uint32_t* thr = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)r->n_levels);
  if (!fl || !thr) {
    free(fl);
    free(thr);
    return OR_ERR_NOMEM;
  }
  set_threads(r);
  for (int32_t p = 0; p < r->cfg.n_pop; ++p) {
    or_pop* P = &r->pops[p];
    or_obs* o = obs_at(r, t, p);
    /* 1. reweighting factors from the energy levels of the step t-1 population */
    const int64_t* cprev = hist_at(r, t - 1, p);
    double S, eps;
    int32_t kmin = or_reweight(r->n_levels, cprev, r->cfg.R, dbeta, &S, fl, thr, &eps);
    if (kmin < 0) {
      free(fl);
      free(thr);
      return OR_ERR_INVALID;
    }
    /* 2. copy numbers n_i, nearest-integer rule */
    const int32_t* Eold = P->E[P->cur];
    int64_t newR = 0, culled = 0;
    for (int64_t i = 0; i < P->Rt; ++i) {
      int32_t k = (Eold[i] + 3 * N) / 2;
      int32_t n = or_copy_count(r->cfg.run_seed, p, t, i, fl[k], thr[k]);
      P->counts[i] = n;
      newR += n;
      if (n == 0) culled += 1;
    }
    P->counts_n = P->Rt;
    if (newR > r->cfg.R_cap) {
      free(fl);
      free(thr);
      return OR_ERR_CAPACITY;
    }
    if (newR == 0) {
      free(fl);
      free(thr);
      return OR_ERR_INVALID;
    }
    /* 3. the new population: n_i copies of replica i, in slot order; each copy
     * inherits the family label (§II) */
    int nxt = 1 - P->cur;
    int64_t j = 0;
    for (int64_t i = 0; i < P->Rt; ++i)
      for (int32_t q = 0; q < P->counts[i]; ++q, ++j) {
        memcpy(P->s[nxt] + (size_t)j * N, P->s[P->cur] + (size_t)i * N, (size_t)N);
        P->lab[nxt][j] = P->lab[P->cur][i];
        P->E[nxt][j] = Eold[i];
      }
    /* 4. ln Q(beta_{t-1}, beta_t) = ln(S'/R~_{t-1}) - dbeta E_min (Eq. Q) */
    int32_t Emin_prev = 2 * kmin - 3 * N;
    double lnQ = log(S / (double)P->Rt) - dbeta * (double)Emin_prev;
    P->lnQ_sum = P->lnQ_sum + lnQ;
    P->cur = nxt;
    P->Rt = newR;
    /* 5. Metropolis sweeps at beta_t */
    int8_t* s = P->s[P->cur];
    int32_t* E = P->E[P->cur];
    int32_t S_t = r->sweeps[t];
#pragma omp parallel for schedule(static)
    for (int64_t jj = 0; jj < newR; ++jj)
      E[jj] += or_sweep_replica(r->L, r->J, s + (size_t)jj * N, r->cfg.run_seed, p, jj, t, S_t, met);
    o->dbeta = dbeta;
    o->kmin_prev = kmin;
    o->S_prime = S;
    o->lnQ = lnQ;
    o->eps_expected = eps;
    o->culled = culled;
  }
  free(fl);
  free(thr);
  /* 6. measure */
  int rc = measure(r, t);
  if (rc != OR_OK) return rc;
  r->t = t;
  if (t == r->cfg.n_temps - 1 || (!r->cfg.betas && r->betas[t] >= r->cfg.beta_max)) r->done = 1;
  return OR_OK;
}

int or_run_all(or_run* r) {
  int rc;
  while ((rc = or_step(r)) == OR_OK) {
  }
  return rc == OR_DONE ? OR_OK : rc;
}

int32_t or_current_step(const or_run* r) { return r->t; }
double or_beta(const or_run* r, int32_t t) { return (t >= 0 && t <= r->t) ? r->betas[t] : -1.0; }
const int8_t* or_couplings_of(const or_run* r) { return r->J; }

int or_observables(const or_run* r, int32_t t, int32_t pop, or_obs* out) {
  if (t < 0 || t > r->t || pop < 0 || pop >= r->cfg.n_pop) return OR_ERR_INVALID;
  *out = *obs_at(r, t, pop);
  return OR_OK;
}

int or_energy_hist(const or_run* r, int32_t t, int32_t pop, int64_t* out) {
  if (t < 0 || t > r->t || pop < 0 || pop >= r->cfg.n_pop) return OR_ERR_INVALID;
  memcpy(out, hist_at(r, t, pop), sizeof(int64_t) * (size_t)r->n_levels);
  return OR_OK;
}

int or_q_hist(const or_run* r, int32_t t, int64_t* out) {
  if (t < 0 || t > r->t || r->cfg.n_pop != 2) return OR_ERR_INVALID;
  memcpy(out, &r->qhist[(size_t)t * r->cfg.q_bins], sizeof(int64_t) * (size_t)r->cfg.q_bins);
  return OR_OK;
}

int or_family_hist(const or_run* r, int32_t pop, int64_t cap, int64_t* eta, int64_t* m, int64_t* n) {
  if (pop < 0 || pop >= r->cfg.n_pop) return OR_ERR_INVALID;
  const or_pop* P = &r->pops[pop];
  const int32_t* lab = P->lab[P->cur];
  int64_t R = P->Rt;
  int64_t* cnt = (int64_t*)calloc((size_t)R + 1, sizeof(int64_t));
  if (!cnt) return OR_ERR_NOMEM;
  int64_t start = 0;
  for (int64_t j = 1; j <= R; ++j)
    if (j == R || lab[j] != lab[start]) {
      cnt[j - start] += 1;
      start = j;
    }
  int64_t k = 0;
  for (int64_t e = 1; e <= R; ++e)
    if (cnt[e] > 0) {
      if (k < cap) {
        eta[k] = e;
        m[k] = cnt[e];
      }
      ++k;
    }
  free(cnt);
  *n = k;
  return k <= cap ? OR_OK : OR_ERR_CAPACITY;
}

int or_population(const or_run* r, int32_t pop, int64_t cap, int8_t* spins, int32_t* labels,
                  int32_t* energies, int64_t* count) {
  if (pop < 0 || pop >= r->cfg.n_pop) return OR_ERR_INVALID;
  const or_pop* P = &r->pops[pop];
  *count = P->Rt;
  if (P->Rt > cap) return OR_ERR_CAPACITY;
  if (spins) memcpy(spins, P->s[P->cur], (size_t)P->Rt * r->N);
  if (labels) memcpy(labels, P->lab[P->cur], sizeof(int32_t) * (size_t)P->Rt);
  if (energies) memcpy(energies, P->E[P->cur], sizeof(int32_t) * (size_t)P->Rt);
  return OR_OK;
}

int or_last_counts(const or_run* r, int32_t pop, int64_t cap, int32_t* counts, int64_t* count) {
  if (pop < 0 || pop >= r->cfg.n_pop || r->t == 0) return OR_ERR_INVALID;
  const or_pop* P = &r->pops[pop];
  *count = P->counts_n;
  if (P->counts_n > cap) return OR_ERR_CAPACITY;
  memcpy(counts, P->counts, sizeof(int32_t) * (size_t)P->counts_n);
  return OR_OK;
}

void or_destroy(or_run* r) { free_run(r); }
