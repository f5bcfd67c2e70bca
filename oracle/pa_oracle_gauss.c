/* pa_oracle_gauss.c — plain CPU oracle for population annealing on the 3D
 * Edwards-Anderson spin glass with GAUSSIAN couplings (the paper's model, §II.A).
 *
 * TEST INFRASTRUCTURE ONLY (see pa_oracle.h).  Written step by step from the
 * paper; it shares nothing with the CUDA library.
 *
 * Readings, so that every floating-point decision has one definition:
 *   - J(n,d) ~ N(0,1) by Box-Muller from Philox words at counter (n, 1, 0, 0),
 *     clamped to [-5, 5] and held in fixed point, Jq = round(J * 2^20); energies
 *     and energy changes are then exact integers (units of 2^-20);
 *   - a Metropolis flip with dE <= 0 is taken; otherwise it is taken when the
 *     replica's 32-bit uniform U < thr(dE) = min(floor(2^32 exp(-beta dE)),
 *     2^32 - 2), the exponential in double precision (2^32 p is then exact, a
 *     power-of-two scaling, and the floor the only rounding).  U is a random-stream
 *     convention (the paper fixes no generator): its upper 16 bits are half
 *     (slot & 1) of word (slot >> 1) & 3 of Philox at counter
 *     (n >> 1, 2 sweep + colour, slot >> 3, t), its lower 16 bits the upper half of
 *     word slot & 3 of Philox at counter (n >> 1, 2 sweep + colour,
 *     (slot >> 2) | 2^31, t) (org_metropolis_uniform);
 *   - resampling follows Eqs. (tau), (Q) and (eq_num_elim) as written, replica by
 *     replica: each weight is one exponential, w_i = exp(-dbeta (E_i - E_min)) with
 *     E_min the lowest energy present (Eq. Q divided by its largest term); S' is
 *     the sum of the weights in slot order, tau_i = R w_i / S', and the culling sum
 *     adds 1 - tau_i over the replicas with tau_i < 1, again in slot order;
 *   - the adaptive schedule (§IV.B) bisects on that culling fraction.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#include "pa_oracle.h"

#define JSCALE_LOG2 20
#define JCLAMP 5.0

static int32_t g_site(int32_t L, int32_t x, int32_t y, int32_t z) {
  x = (x % L + L) % L;
  y = (y % L + L) % L;
  z = (z % L + L) % L;
  return x + L * (y + L * z);
}

static int32_t g_neighbour(int32_t L, int32_t n, int32_t d, int32_t dir) {
  int32_t x = n % L, y = (n / L) % L, z = n / (L * L);
  if (d == 0) x += dir;
  if (d == 1) y += dir;
  if (d == 2) z += dir;
  return g_site(L, x, y, z);
}

static uint32_t g_word(const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int which) {
  uint32_t ctr[4] = {c0, c1, c2, c3}, out[4];
  or_philox4x32_10(ctr, key, out);
  return out[which];
}

/* ---- couplings and energy ---- */

static int32_t quantise(double g) {
  if (g > JCLAMP) g = JCLAMP;
  if (g < -JCLAMP) g = -JCLAMP;
  return (int32_t)llround(g * 1048576.0);
}

void org_couplings(int32_t L, uint64_t disorder_seed, int32_t* Jq) {
  int32_t N = L * L * L;
  uint32_t key[2], w[4];
  or_key(disorder_seed, OR_P_COUPLINGS, 0, key);
  for (int32_t n = 0; n < N; ++n) {
    uint32_t ctr[4] = {(uint32_t)n, 1u, 0u, 0u};
    or_philox4x32_10(ctr, key, w);
    double u1 = ((double)w[0] + 0.5) * 0x1p-32, u2 = ((double)w[1] + 0.5) * 0x1p-32;
    double u3 = ((double)w[2] + 0.5) * 0x1p-32, u4 = ((double)w[3] + 0.5) * 0x1p-32;
    double ra = sqrt(-2.0 * log(u1)), rb = sqrt(-2.0 * log(u3));
    double ta = (2.0 * M_PI) * u2, tb = (2.0 * M_PI) * u4;
    Jq[3 * n + 0] = quantise(ra * cos(ta));
    Jq[3 * n + 1] = quantise(ra * sin(ta));
    Jq[3 * n + 2] = quantise(rb * cos(tb));
  }
}

int64_t org_energy(int32_t L, const int32_t* Jq, const int8_t* s) {
  int32_t N = L * L * L;
  int64_t E = 0;
  for (int32_t n = 0; n < N; ++n)
    for (int32_t d = 0; d < 3; ++d) E -= (int64_t)Jq[3 * n + d] * s[n] * s[g_neighbour(L, n, d, +1)];
  return E;
}

/* ---- Metropolis ---- */

/* Energy change of flipping s_n: dE = 2 s_n sum_m J_nm s_m over its six bonds. */
static int64_t flip_change(int32_t L, const int32_t* Jq, const int8_t* s, int32_t n) {
  int32_t xp = g_neighbour(L, n, 0, +1), xm = g_neighbour(L, n, 0, -1);
  int32_t yp = g_neighbour(L, n, 1, +1), ym = g_neighbour(L, n, 1, -1);
  int32_t zp = g_neighbour(L, n, 2, +1), zm = g_neighbour(L, n, 2, -1);
  int64_t h = (int64_t)Jq[3 * n + 0] * s[xp] + (int64_t)Jq[3 * xm + 0] * s[xm] + (int64_t)Jq[3 * n + 1] * s[yp] +
              (int64_t)Jq[3 * ym + 1] * s[ym] + (int64_t)Jq[3 * n + 2] * s[zp] + (int64_t)Jq[3 * zm + 2] * s[zm];
  return 2 * s[n] * h;
}

uint32_t org_metropolis_uniform(uint64_t run_seed, int32_t pop, int32_t n, int32_t sweep, int32_t colour,
                                int64_t slot, int32_t t) {
  uint32_t key[2];
  or_key(run_seed, OR_P_METROPOLIS, (uint32_t)pop, key);
  const uint32_t q = (uint32_t)(2 * sweep + colour), h = (uint32_t)(n >> 1);
  const uint32_t upper_word = g_word(key, h, q, (uint32_t)(slot >> 3), (uint32_t)t, (int)((slot >> 1) & 3));
  const uint32_t upper = (slot & 1) ? upper_word >> 16 : upper_word & 0xffffu;
  const uint32_t lower_word =
      g_word(key, h, q, (uint32_t)(slot >> 2) | 0x80000000u, (uint32_t)t, (int)(slot & 3));
  return (upper << 16) | (lower_word >> 16);
}

uint32_t org_acceptance_threshold(double beta, int64_t dE) {
  double v = floor(exp(-(beta * ((double)dE * 0x1p-20))) * 4294967296.0);
  if (v > 4294967294.0) v = 4294967294.0;
  return (uint32_t)v;
}

int64_t org_sweep_replica(int32_t L, const int32_t* Jq, int8_t* s, uint64_t run_seed, int32_t pop, int64_t slot,
                          int32_t t, int32_t n_sweeps, double beta) {
  int64_t total = 0;
  for (int32_t sw = 0; sw < n_sweeps; ++sw)
    for (int32_t c = 0; c < 2; ++c)
      for (int32_t z = 0; z < L; ++z)
        for (int32_t y = 0; y < L; ++y)
          for (int32_t x = 0; x < L; ++x) {
            if ((x + y + z) % 2 != c) continue;
            int32_t n = g_site(L, x, y, z);
            int64_t dE = flip_change(L, Jq, s, n);
            if (dE <= 0 || org_metropolis_uniform(run_seed, pop, n, sw, c, slot, t) < org_acceptance_threshold(beta, dE)) {
              s[n] = (int8_t)(-s[n]);
              total += dE;
            }
          }
  return total;
}

/* ---- resampling, §II Eqs. (tau), (Q) and (eq_num_elim) ---- */

/* Weight of a replica whose energy lies d above the lowest one (fixed point,
 * units of 2^-20): exp(-dbeta (E - E_min)). */
double org_weight(double dbeta, int64_t d) { return exp(-(dbeta * ((double)d * 0x1p-20))); }

/* The reweighting of a population of n replicas with energies E to a temperature
 * dbeta lower: E_min, S' = sum_i w_i (slot order), the expected culling fraction
 * (1/R) sum_{tau_i < 1} (1 - tau_i) (slot order), and tau_i = R w_i / S' when tau
 * is not NULL.  Returns OR_ERR_INVALID for an empty population. */
int org_reweight(const int64_t* E, int64_t n, int64_t R, double dbeta, int64_t* E_min, double* S_prime,
                 double* eps_expected, double* tau) {
  if (n < 1) return OR_ERR_INVALID;
  int64_t Emin = E[0];
  for (int64_t i = 1; i < n; ++i)
    if (E[i] < Emin) Emin = E[i];
  double S = 0.0;
  for (int64_t i = 0; i < n; ++i) S = S + org_weight(dbeta, E[i] - Emin);
  double cull = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double t_i = ((double)R * org_weight(dbeta, E[i] - Emin)) / S;
    if (t_i < 1.0) cull = cull + (1.0 - t_i);
    if (tau) tau[i] = t_i;
  }
  *E_min = Emin;
  *S_prime = S;
  *eps_expected = cull / (double)R;
  return OR_OK;
}

/* ---- the run (§II), explicit schedules ---- */

typedef struct {
  int8_t* s[2];
  int32_t* lab[2];
  int64_t* E[2];
  int cur;
  int64_t Rt;
  int32_t* counts;
  int64_t counts_n;
  int64_t E0;
  double lnQ_sum;
} org_pop;

struct org_run {
  or_config cfg;
  int32_t L, N;
  int32_t* Jq;
  double* betas;
  int32_t* sweeps;
  int32_t t;
  int done;
  org_pop pops[2];
  org_obs* obs;      /* [n_temps][n_pop] */
  int64_t* qhist;    /* [n_temps][q_bins] spin overlap */
  int64_t* qlhist;   /* [n_temps][q_bins] link overlap */
};

static org_obs* gobs_at(const org_run* r, int32_t t, int32_t p) { return &r->obs[(size_t)t * r->cfg.n_pop + p]; }

static int family_stats_g(const org_pop* P, int64_t* sum_eta2, int64_t* n_fam, double* S_f, int64_t* mh) {
  const int32_t* lab = P->lab[P->cur];
  int64_t R = P->Rt, s2 = 0, nf = 0, start = 0;
  memset(mh, 0, sizeof(int64_t) * (size_t)(R + 1));
  for (int64_t j = 1; j <= R; ++j)
    if (j == R || lab[j] != lab[start]) {
      if (j < R && lab[j] < lab[start]) return OR_ERR_INVALID;
      int64_t eta = j - start;
      s2 += eta * eta;
      nf += 1;
      mh[eta] += 1;
      start = j;
    }
  double S = 0.0;
  for (int64_t eta = 1; eta <= R; ++eta) {
    if (mh[eta] == 0) continue;
    double nu = (double)eta / (double)R;
    S = S - (double)mh[eta] * (nu * log(nu));
  }
  *sum_eta2 = s2;
  *n_fam = nf;
  *S_f = S;
  return OR_OK;
}

static int measure_g(org_run* r, int32_t t) {
  int32_t N = r->N;
  for (int32_t p = 0; p < r->cfg.n_pop; ++p) {
    org_pop* P = &r->pops[p];
    const int64_t* E = P->E[P->cur];
    int64_t sE = 0, Emin = INT64_MAX;
    __int128 sE2 = 0;
    for (int64_t j = 0; j < P->Rt; ++j) {
      sE += E[j];
      sE2 += (__int128)E[j] * E[j];
      if (E[j] < Emin) Emin = E[j];
    }
    if (t == 0 || Emin < P->E0) P->E0 = Emin;
    int64_t at0 = 0;
    for (int64_t j = 0; j < P->Rt; ++j) at0 += E[j] == P->E0;
    org_obs* o = gobs_at(r, t, p);
    o->t = t;
    o->beta = r->betas[t];
    o->R_tilde = P->Rt;
    o->sum_E = sE;
    o->sum_E2 = (double)sE2;
    o->E_min = Emin;
    o->mean_E = ((double)sE / (double)P->Rt) * 0x1p-20;
    o->var_E = (o->sum_E2 / (double)P->Rt) * 0x1p-40 - o->mean_E * o->mean_E;
    o->minus_beta_F = (double)N * log(2.0) + P->lnQ_sum;
    o->E0 = P->E0;
    o->g0_tilde = (double)at0 / (double)P->Rt;
    o->g0_bar = 2.0 * exp(-(o->beta * ((double)P->E0 * 0x1p-20)) - o->minus_beta_F);
    int64_t* mh = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P->Rt + 1));
    if (!mh) return OR_ERR_NOMEM;
    int rc = family_stats_g(P, &o->sum_eta2, &o->n_families, &o->S_f, mh);
    free(mh);
    if (rc != OR_OK) return rc;
    o->rho_t = (double)o->sum_eta2 / (double)P->Rt;
    o->rho_s = (double)P->Rt / exp(o->S_f);
    o->q_pairs = 0;
    o->q_abs_le_02 = 0;
    o->I02 = 0.0;
    o->ql_sum = 0;
    o->ql_mean = 0.0;
    o->e_l = 0.0;
    o->delta_KY = 0.0;
  }
  if (r->cfg.n_pop == 2) {
    /* spin overlap q (§II.A) and link overlap q_l = (1/N_b) sum over bonds of
     * s1_n s1_m s2_n s2_m (Eq. ql), between slot j of the two populations */
    int64_t* qh = &r->qhist[(size_t)t * r->cfg.q_bins];
    int64_t* qlh = &r->qlhist[(size_t)t * r->cfg.q_bins];
    memset(qh, 0, sizeof(int64_t) * (size_t)r->cfg.q_bins);
    memset(qlh, 0, sizeof(int64_t) * (size_t)r->cfg.q_bins);
    const org_pop* A = &r->pops[0];
    const org_pop* B = &r->pops[1];
    int64_t pairs = A->Rt < B->Rt ? A->Rt : B->Rt;
    int64_t small = 0, ql_sum = 0, nb = r->cfg.q_bins, Nb = 3 * (int64_t)N;
    for (int64_t j = 0; j < pairs; ++j) {
      const int8_t* sa = A->s[A->cur] + (size_t)j * N;
      const int8_t* sb = B->s[B->cur] + (size_t)j * N;
      int64_t Q = 0, QL = 0;
      for (int32_t n = 0; n < N; ++n) Q += sa[n] * sb[n];
      for (int32_t n = 0; n < N; ++n)
        for (int32_t d = 0; d < 3; ++d) {
          int32_t m = g_neighbour(r->L, n, d, +1);
          QL += sa[n] * sa[m] * sb[n] * sb[m];
        }
      qh[((Q + N) * (nb - 1) + N) / (2 * (int64_t)N)] += 1;
      qlh[((QL + Nb) * (nb - 1) + Nb) / (2 * Nb)] += 1;
      if (5 * (Q < 0 ? -Q : Q) <= N) small += 1;
      ql_sum += QL;
    }
    for (int32_t p = 0; p < 2; ++p) {
      org_obs* o = gobs_at(r, t, p);
      o->q_pairs = pairs;
      o->q_abs_le_02 = small;
      o->I02 = pairs > 0 ? (double)small / (double)pairs : 0.0;
      o->ql_sum = ql_sum;
      o->ql_mean = pairs > 0 ? (double)ql_sum / ((double)Nb * (double)pairs) : 0.0;
      /* Eq. (el): e_l = -(1/T)(N_b/N)(1 - <q_l>); Delta_KY for this sample = e_l - e */
      o->e_l = -(o->beta * 3.0) * (1.0 - o->ql_mean);
      o->delta_KY = o->e_l - o->mean_E / (double)N;
    }
  }
  return OR_OK;
}

static void free_g(org_run* r) {
  if (!r) return;
  for (int p = 0; p < 2; ++p) {
    for (int b = 0; b < 2; ++b) {
      free(r->pops[p].s[b]);
      free(r->pops[p].lab[b]);
      free(r->pops[p].E[b]);
    }
    free(r->pops[p].counts);
  }
  free(r->Jq);
  free(r->betas);
  free(r->sweeps);
  free(r->obs);
  free(r->qhist);
  free(r->qlhist);
  free(r);
}

int org_create(const or_config* cfg, org_run** out) {
  *out = NULL;
  if (!cfg || cfg->L < 2 || cfg->L % 2 != 0 || cfg->R < 1 || cfg->n_temps < 1 || cfg->n_pop < 1 || cfg->n_pop > 2 ||
      cfg->q_bins < 3 || cfg->disorder_seed >= ((uint64_t)1 << 56) ||
      cfg->run_seed >= ((uint64_t)1 << 56) || cfg->R_cap < cfg->R || cfg->R_cap >= ((int64_t)1 << 31))
    return OR_ERR_INVALID;
  if (!cfg->betas && !(cfg->eps_target > 0.0 && cfg->eps_target < 1.0 && cfg->beta_max > 0.0))
    return OR_ERR_INVALID;
  if (cfg->betas) {
    if (cfg->betas[0] != 0.0) return OR_ERR_INVALID;
    for (int32_t t = 1; t < cfg->n_temps; ++t)
      if (!(cfg->betas[t] >= cfg->betas[t - 1])) return OR_ERR_INVALID;
  }
  org_run* r = (org_run*)calloc(1, sizeof(org_run));
  if (!r) return OR_ERR_NOMEM;
  r->cfg = *cfg;
  r->L = cfg->L;
  r->N = cfg->L * cfg->L * cfg->L;
  int32_t N = r->N, T = cfg->n_temps;
  r->Jq = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)N);
  r->betas = (double*)calloc((size_t)T, sizeof(double));
  r->sweeps = (int32_t*)calloc((size_t)T, sizeof(int32_t));
  r->obs = (org_obs*)calloc((size_t)T * cfg->n_pop, sizeof(org_obs));
  r->qhist = (int64_t*)calloc((size_t)T * cfg->q_bins, sizeof(int64_t));
  r->qlhist = (int64_t*)calloc((size_t)T * cfg->q_bins, sizeof(int64_t));
  if (!r->Jq || !r->betas || !r->sweeps || !r->obs || !r->qhist || !r->qlhist) {
    free_g(r);
    return OR_ERR_NOMEM;
  }
  for (int32_t t = 0; t < T; ++t) {
    r->betas[t] = cfg->betas ? cfg->betas[t] : 0.0;
    r->sweeps[t] = cfg->sweeps_per_step ? cfg->sweeps_per_step[t] : cfg->n_sweeps;
  }
  r->cfg.betas = cfg->betas ? r->betas : NULL; /* non-NULL marks an explicit schedule */
  r->cfg.sweeps_per_step = NULL;
  org_couplings(r->L, cfg->disorder_seed, r->Jq);
  for (int32_t p = 0; p < cfg->n_pop; ++p) {
    org_pop* P = &r->pops[p];
    for (int b = 0; b < 2; ++b) {
      P->s[b] = (int8_t*)malloc((size_t)cfg->R_cap * N);
      P->lab[b] = (int32_t*)malloc(sizeof(int32_t) * (size_t)cfg->R_cap);
      P->E[b] = (int64_t*)malloc(sizeof(int64_t) * (size_t)cfg->R_cap);
      if (!P->s[b] || !P->lab[b] || !P->E[b]) {
        free_g(r);
        return OR_ERR_NOMEM;
      }
    }
    P->counts = (int32_t*)malloc(sizeof(int32_t) * (size_t)cfg->R_cap);
    if (!P->counts) {
      free_g(r);
      return OR_ERR_NOMEM;
    }
    P->Rt = cfg->R;
    uint32_t key[2];
    or_key(cfg->run_seed, OR_P_INIT, (uint32_t)p, key);
    for (int64_t j = 0; j < cfg->R; ++j) {
      for (int32_t n = 0; n < N; ++n) {
        uint32_t w = g_word(key, (uint32_t)n, 0, (uint32_t)(j >> 2), 0, (int)(j & 3));
        P->s[0][(size_t)j * N + n] = (w & 1u) == 0 ? 1 : -1;
      }
      P->lab[0][j] = (int32_t)j;
      P->E[0][j] = org_energy(r->L, r->Jq, P->s[0] + (size_t)j * N);
    }
  }
  int rc = measure_g(r, 0);
  if (rc != OR_OK) {
    free_g(r);
    return rc;
  }
  r->done = T == 1 || (!cfg->betas && cfg->beta_max <= 0.0);
  *out = r;
  return OR_OK;
}

/* Expected culling fraction (Eq. eq_num_elim / R) of a move by dbeta from population p. */
static double eps_g(const org_run* r, const org_pop* P, double dbeta) {
  int64_t Emin;
  double S, eps;
  org_reweight(P->E[P->cur], P->Rt, r->cfg.R, dbeta, &Emin, &S, &eps, NULL);
  return eps;
}

/* Adaptive step (§IV.B), as for +-1 couplings: the largest dbeta in
 * (0, beta_max - beta] whose culling fraction does not exceed the target, by 64
 * bisection halvings; population 0 decides. */
static void choose_dbeta_g(const org_run* r, int32_t t, double* dbeta) {
  const org_pop* P = &r->pops[0];
  double rem = r->cfg.beta_max - r->betas[t - 1];
  if (eps_g(r, P, rem) <= r->cfg.eps_target) {
    *dbeta = rem;
    return;
  }
  double lo = 0.0, hi = rem;
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi);
    if (eps_g(r, P, mid) <= r->cfg.eps_target)
      lo = mid;
    else
      hi = mid;
  }
  *dbeta = lo > 0.0 ? lo : hi;
}

int org_step(org_run* r) {
  if (r->done) return OR_DONE;
  int32_t t = r->t + 1, N = r->N;
  double dbeta;
  if (r->cfg.betas) {
    dbeta = r->betas[t] - r->betas[t - 1];
  } else {
    choose_dbeta_g(r, t, &dbeta);
    double b = r->betas[t - 1] + dbeta;
    if (b >= r->cfg.beta_max || dbeta == r->cfg.beta_max - r->betas[t - 1]) b = r->cfg.beta_max;
    r->betas[t] = b;
  }
  for (int32_t p = 0; p < r->cfg.n_pop; ++p) {
    org_pop* P = &r->pops[p];
    org_obs* o = gobs_at(r, t, p);
    const int64_t* Eold = P->E[P->cur];
    int64_t R = P->Rt;
    /* 1. weights measured from the lowest energy (Eq. Q), S' and tau (Eq. tau) */
    double* tau = (double*)malloc(sizeof(double) * (size_t)R);
    if (!tau) return OR_ERR_NOMEM;
    int64_t Emin;
    double S, eps;
    org_reweight(Eold, R, r->cfg.R, dbeta, &Emin, &S, &eps, tau);
    /* 2. copy numbers, nearest-integer rule */
    int64_t newR = 0, culled = 0;
    for (int64_t i = 0; i < R; ++i) {
      double f = floor(tau[i]);
      uint32_t thr = (uint32_t)((tau[i] - f) * 4294967296.0);
      int32_t n = or_copy_count(r->cfg.run_seed, p, t, i, (int32_t)f, thr);
      P->counts[i] = n;
      newR += n;
      culled += n == 0;
    }
    free(tau);
    P->counts_n = R;
    if (newR > r->cfg.R_cap || newR == 0) return newR == 0 ? OR_ERR_INVALID : OR_ERR_CAPACITY;
    /* 3. the new population, copies in slot order with inherited labels */
    int nxt = 1 - P->cur;
    int64_t j = 0;
    for (int64_t i = 0; i < R; ++i)
      for (int32_t q = 0; q < P->counts[i]; ++q, ++j) {
        memcpy(P->s[nxt] + (size_t)j * N, P->s[P->cur] + (size_t)i * N, (size_t)N);
        P->lab[nxt][j] = P->lab[P->cur][i];
        P->E[nxt][j] = Eold[i];
      }
    double lnQ = log(S / (double)R) - dbeta * ((double)Emin * 0x1p-20);
    P->lnQ_sum = P->lnQ_sum + lnQ;
    P->cur = nxt;
    P->Rt = newR;
    /* 4. Metropolis sweeps at beta_t */
    int8_t* s = P->s[P->cur];
    int64_t* E = P->E[P->cur];
#pragma omp parallel for schedule(static)
    for (int64_t jj = 0; jj < newR; ++jj)
      E[jj] += org_sweep_replica(r->L, r->Jq, s + (size_t)jj * N, r->cfg.run_seed, p, jj, t, r->sweeps[t],
                                 r->betas[t]);
    o->dbeta = dbeta;
    o->E_min_prev = Emin;
    o->S_prime = S;
    o->lnQ = lnQ;
    o->eps_expected = eps;
    o->culled = culled;
  }
  int rc = measure_g(r, t);
  if (rc != OR_OK) return rc;
  r->t = t;
  if (t == r->cfg.n_temps - 1 || (!r->cfg.betas && r->betas[t] >= r->cfg.beta_max)) r->done = 1;
  return OR_OK;
}

int org_run_all(org_run* r) {
  int rc;
  while ((rc = org_step(r)) == OR_OK) {
  }
  return rc == OR_DONE ? OR_OK : rc;
}

int32_t org_current_step(const org_run* r) { return r->t; }

int org_observables(const org_run* r, int32_t t, int32_t pop, org_obs* out) {
  if (t < 0 || t > r->t || pop < 0 || pop >= r->cfg.n_pop) return OR_ERR_INVALID;
  *out = *gobs_at(r, t, pop);
  return OR_OK;
}

int org_q_hist(const org_run* r, int32_t t, int32_t link, int64_t* out) {
  if (t < 0 || t > r->t || r->cfg.n_pop != 2) return OR_ERR_INVALID;
  memcpy(out, (link ? r->qlhist : r->qhist) + (size_t)t * r->cfg.q_bins, sizeof(int64_t) * (size_t)r->cfg.q_bins);
  return OR_OK;
}

int org_population(const org_run* r, int32_t pop, int64_t cap, int8_t* spins, int32_t* labels, int64_t* E,
                   int64_t* n) {
  if (pop < 0 || pop >= r->cfg.n_pop) return OR_ERR_INVALID;
  const org_pop* P = &r->pops[pop];
  *n = P->Rt;
  if (P->Rt > cap) return OR_ERR_CAPACITY;
  memcpy(spins, P->s[P->cur], (size_t)P->Rt * r->N);
  memcpy(labels, P->lab[P->cur], sizeof(int32_t) * (size_t)P->Rt);
  memcpy(E, P->E[P->cur], sizeof(int64_t) * (size_t)P->Rt);
  return OR_OK;
}

int org_last_counts(const org_run* r, int32_t pop, int64_t cap, int32_t* counts, int64_t* n) {
  if (pop < 0 || pop >= r->cfg.n_pop) return OR_ERR_INVALID;
  const org_pop* P = &r->pops[pop];
  *n = P->counts_n;
  if (P->counts_n > cap) return OR_ERR_CAPACITY;
  memcpy(counts, P->counts, sizeof(int32_t) * (size_t)P->counts_n);
  return OR_OK;
}

const int32_t* org_couplings_of(const org_run* r) { return r->Jq; }

void org_destroy(org_run* r) { free_g(r); }
