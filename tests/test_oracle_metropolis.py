"""Pin for the oracle's checkerboard Metropolis sweep (§II, MCMC at fixed beta).

A population resampled once from beta = 0 to beta and then swept many times is
a set of independent Metropolis chains; its energy histogram must follow the
exact Boltzmann distribution g(k) exp(-beta E_k) / Z from enumeration.  L = 2
(two-colour) and L = 3 (three-colour) are both covered.
"""
import numpy as np
import pytest
from scipy import stats


def boltzmann_levels(L, g, beta):
    N = L ** 3
    k = np.arange(3 * N + 1)
    E = 2 * k - 3 * N
    logw = np.where(g > 0, np.log(np.maximum(g, 1)) - beta * E, -np.inf)
    p = np.exp(logw - logw.max())
    return p / p.sum()


def chi2_pvalue(observed, p, min_expected=5.0):
    n = observed.sum()
    e = n * p
    keep = e >= min_expected
    obs = list(observed[keep]) + [observed[~keep].sum()]
    exp_ = list(e[keep]) + [e[~keep].sum()]
    obs, exp_ = np.array(obs, float), np.array(exp_, float)
    if exp_[-1] < min_expected:
        obs[-2] += obs[-1]
        exp_[-2] += exp_[-1]
        obs, exp_ = obs[:-1], exp_[:-1]
    chi2 = ((obs - exp_) ** 2 / exp_).sum()
    return stats.chi2.sf(chi2, len(obs) - 1)


@pytest.mark.parametrize("L,R,beta,seed", [(2, 20000, 0.4, 5), (2, 20000, 0.9, 6), (3, 6000, 0.5, 7),
                                           (3, 6000, 1.1, 8)])
def test_sweeps_sample_boltzmann(oracle_lib, L, R, beta, seed):
    run = oracle_lib.Run(oracle_lib.RunConfig(L=L, R=R, disorder_seed=seed, run_seed=100 + seed,
                                              betas=np.array([0.0, beta]), n_sweeps=0,
                                              sweeps_per_step=np.array([0, 100], dtype=np.int32)))
    run.run()
    J = run.couplings()
    g = oracle_lib.enumerate_levels(L, J)
    c = run.energy_hist(1)
    assert c.sum() == run.obs(1)["R_tilde"]
    p = boltzmann_levels(L, g, beta)
    assert chi2_pvalue(c, p) > 1e-6
    # every stored energy equals the energy of the stored spins
    s, _, E = run.population()
    for j in range(0, len(E), max(1, len(E) // 200)):
        assert oracle_lib.energy(L, J, s[j]) == E[j]


def test_sweep_replica_is_deterministic_and_seeded(oracle_lib):
    L = 4
    J = oracle_lib.couplings(L, 1)
    s0 = np.where(np.random.default_rng(0).random(L ** 3) < 0.5, 1, -1).astype(np.int8)
    thr = oracle_lib.metropolis_thresholds(0.8)
    a, dEa = oracle_lib.sweep_replica(L, J, s0, 99, 0, 5, 3, 4, thr)
    b, dEb = oracle_lib.sweep_replica(L, J, s0, 99, 0, 5, 3, 4, thr)
    assert np.array_equal(a, b) and dEa == dEb
    assert oracle_lib.energy(L, J, a) - oracle_lib.energy(L, J, s0) == dEa
    c, _ = oracle_lib.sweep_replica(L, J, s0, 99, 0, 6, 3, 4, thr)   # another slot: another stream
    assert not np.array_equal(a, c)
    # beta -> infinity: only dE <= 0 moves are taken, so the energy never rises
    z, dEz = oracle_lib.sweep_replica(L, J, s0, 99, 0, 5, 3, 4, oracle_lib.metropolis_thresholds(60.0))
    assert dEz <= 0


def test_bitwise_test_is_the_comparison_of_the_whole_uniform(oracle_lib):
    """The sweep's test reads the uniform from its top bit and stops at the first bit
    that differs from the threshold; that must be exactly uniform < thr, also for
    thresholds equal to the uniform, one off, 0 and 2^32 - 1."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        seed, pop, site, hs, slot, t = (int(rng.integers(1, 2 ** 40)), int(rng.integers(0, 2)),
                                        int(rng.integers(0, 2 ** 15)), int(rng.integers(0, 40)),
                                        int(rng.integers(0, 10 ** 6)), int(rng.integers(0, 200)))
        r = oracle_lib.metropolis_uniform(seed, pop, site, hs, slot, t)
        for thr in {0, 1, 0xFFFFFFFF, r, max(r - 1, 0), min(r + 1, 0xFFFFFFFF), r ^ 0x80000000, r >> 7,
                    int(rng.integers(0, 2 ** 32))}:
            assert oracle_lib.metropolis_test(seed, pop, site, hs, slot, t, thr) == (r < thr), (r, thr)


def test_bit_column_uniforms_are_uniform_and_independent_between_slots(oracle_lib):
    """The uniforms of the 32 slots that share the stream's words are bit columns of
    the same Philox blocks: each must still be uniform (Kolmogorov-Smirnov) and
    uncorrelated with its neighbours in the word, and slot 32 (the next group of
    blocks) and the next half-sweep must give other numbers."""
    n = 400
    u = np.array([[oracle_lib.metropolis_uniform(77, 0, site, 3, slot, 5) for slot in range(34)]
                  for site in range(n)], dtype=np.float64) / 2.0 ** 32
    for slot in (0, 1, 13, 31, 32, 33):
        assert stats.kstest(u[:, slot], "uniform").pvalue > 1e-4
    for a, b in ((0, 1), (5, 6), (30, 31), (31, 32), (0, 32)):
        assert abs(np.corrcoef(u[:, a], u[:, b])[0, 1]) < 5 / np.sqrt(n)
    assert oracle_lib.metropolis_uniform(77, 0, 9, 3, 0, 5) != oracle_lib.metropolis_uniform(77, 0, 9, 4, 0, 5)
    assert oracle_lib.metropolis_uniform(77, 0, 9, 3, 0, 5) != oracle_lib.metropolis_uniform(77, 1, 9, 3, 0, 5)
