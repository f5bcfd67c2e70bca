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


@pytest.mark.parametrize("thr", [0, 1, 0xFFFF, 0x10000, 0x10001, 0x1234ABCD, 0x8000FFFF, 0xFFFF0000, 0xFFFFFFFE,
                                 0xFFFFFFFF])
def test_two_stage_acceptance_has_the_probability_of_one_32bit_uniform(oracle_lib, thr):
    """Over all 16-bit U (the replica's uniform) and V (its tie-break uniform) the
    rule accepts exactly thr of the 2^32 pairs, i.e. with probability thr / 2^32,
    the same as one 32-bit uniform below thr; and V matters only when U equals
    the top half of thr."""
    accept = oracle_lib.metropolis_accept
    rng = np.random.default_rng(thr & 0xFFFF)
    top = thr >> 16
    total = 0
    for U in range(1 << 16):
        if U == top:
            total += sum(accept(U, V, thr) for V in range(1 << 16))
        else:
            a = accept(U, 0, thr)
            assert a == accept(U, 0xFFFF, thr) == accept(U, int(rng.integers(1 << 16)), thr)
            total += (1 << 16) * a
    assert total == thr
