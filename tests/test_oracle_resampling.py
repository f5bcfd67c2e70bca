"""Pins for the oracle's reweighting and nearest-integer resampling.

Checked against what the paper states and the mathematics fixes:
  * Eqs. (tau), (Q): the expected copy numbers of a population sum to R, and
    their ratios are Boltzmann-factor ratios;
  * §II: n = floor(tau) with probability ceil(tau) - tau, else ceil(tau), so
    E n = tau and var n = f (1 - f), f = frac(tau);
  * Eq. (eps): for Gaussian tau with mean 1 and width sigma, the culled fraction
    is sigma / sqrt(2 pi);
  * Appendix B: sum of var z over a step is 2 eps - 2 pi eps^2 per replica;
  * Eqs. (petak), (rhotb): with energies independent of family, the family
    sizes follow the birth-death law and rho_t - 1 = 2 eps k.
"""
import numpy as np
import pytest


def test_reweight_normalisation_and_ratios(oracle_lib):
    rng = np.random.default_rng(3)
    n_levels = 3 * 4 ** 3 + 1
    c = np.zeros(n_levels, dtype=np.int64)
    c[40:120] = rng.integers(0, 50, size=80)
    R = 1000
    for dbeta in (1e-4, 0.05, 0.3, 2.0):
        kmin, S, fl, thr, eps = oracle_lib.reweight(c, R, dbeta)
        assert kmin == int(np.nonzero(c)[0][0])
        lev = np.arange(kmin, n_levels)
        tau = fl[lev] + thr[lev] / 2.0 ** 32          # tau_k up to 2^-32
        # sum_k c_k tau_k = R (Eq. tau summed over the population)
        assert abs((c[lev] * tau).sum() - R) <= c.sum() * 2.0 ** -32 + 1e-9 * R
        # tau_k / tau_kmin = exp(-dbeta (E_k - E_kmin)), E_k - E_kmin = 2 (k - kmin)
        big = tau > 1e-3
        ratio = tau[big] / tau[0]
        expect = np.exp(-dbeta * 2.0 * (lev[big] - kmin))
        assert np.allclose(ratio, expect, rtol=0, atol=2.0 ** -32 / tau[0] * 4 + 1e-12)
        # Eq. (eq_num_elim) / R
        eps_ref = (c[lev] * np.clip(1 - tau, 0, None)).sum() / R
        assert eps == pytest.approx(eps_ref, abs=c.sum() * 2.0 ** -32 / R + 1e-15)
    assert oracle_lib.reweight(np.zeros(10, dtype=np.int64), 5, 0.1)[0] == -1


@pytest.mark.parametrize("tau", [0.0, 0.3, 1.0, 1.7, 2.45, 5.999, 17.25])
def test_copy_number_law(oracle_lib, tau):
    n = 40000
    counts = oracle_lib.resample_tau(np.full(n, tau), seed=11, t=3)
    f = tau - np.floor(tau)
    assert set(np.unique(counts)) <= {int(np.floor(tau)), int(np.ceil(tau))}
    sd = np.sqrt(f * (1 - f) / n) if 0 < f < 1 else 0.0
    assert abs(counts.mean() - tau) <= 5 * sd + 1e-12
    if 0 < f < 1:
        var = counts.var()
        assert abs(var - f * (1 - f)) < 5 * np.sqrt(f * (1 - f) * (1 - 2 * f) ** 2 / n + 2 * (f * (1 - f)) ** 2 / n) + 1e-3


@pytest.mark.parametrize("sigma", [0.02, 0.08])
def test_gaussian_tau_culling_and_remainder_variance(oracle_lib, sigma):
    rng = np.random.default_rng(int(sigma * 1000))
    n = 200000
    tau = 1.0 + sigma * rng.standard_normal(n)
    eps = sigma / np.sqrt(2 * np.pi)                       # Eq. (eps)
    draws = [oracle_lib.resample_tau(tau, seed=5, t=t) for t in range(4)]
    culled = np.mean([(d == 0).mean() for d in draws])
    assert abs(culled - eps) < 5 * np.sqrt(eps / n / 4) + 5 * sigma / np.sqrt(n)
    # Appendix B: E var z = 2 eps - 2 pi eps^2 (z = n - tau, mean zero)
    z2 = np.mean([((d - tau) ** 2).mean() for d in draws])
    target = 2 * eps - 2 * np.pi * eps ** 2
    assert abs(z2 - target) < 0.03 * target
    for d in draws:
        assert abs(d.sum() - n) < 6 * np.sqrt(n * (2 * eps))


def test_family_size_law_birth_death(oracle_lib):
    """Replicas whose weights are drawn afresh each step (the MCMC-equilibrated
    regime of §III.D): families follow Eq. (petak) and rho_t - 1 = 2 eps k."""
    rng = np.random.default_rng(2024)
    R = 30000
    a = 0.06
    labels = np.arange(R)
    eps_sum = 0.0
    k_steps = 40
    for t in range(1, k_steps + 1):
        w = np.exp(-a * rng.standard_normal(labels.size))
        tau = R * w / w.sum()                               # Eq. (tau)
        eps_sum += np.clip(1 - tau, 0, None).sum() / R      # Eq. (eq_num_elim)
        n = oracle_lib.resample_tau(tau, seed=77, t=t)
        labels = np.repeat(labels, n)
    eps = eps_sum / k_steps
    eta = np.bincount(labels, minlength=R)
    rho_t = (eta.astype(np.float64) ** 2).sum() / R
    ek = eps * k_steps
    assert abs((rho_t - 1) - 2 * ek) < 0.08 * 2 * ek       # Eq. (rhotb)
    P0 = (eta == 0).mean()
    assert abs(P0 - ek / (1 + ek)) < 0.03                  # P_0(k)
    # Eq. (petak): geometric family sizes with ratio ek / (1 + ek)
    for size in (1, 2, 3):
        p = (eta == size).mean()
        expect = (1 / (1 + ek)) ** 2 * (ek / (1 + ek)) ** (size - 1)
        assert abs(p - expect) < 0.15 * expect
