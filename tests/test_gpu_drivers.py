"""The paper's rho_f / rho_t relations and its population-size scheme, on GPU runs.

In the MCMC-equilibrated regime (high temperature, enough sweeps) the paper
derives rho_f = 2 pi sum eps^2 (Eq. rhofgrow), rho_t - 1 = 2 sum eps
(Eq. rhotb) and rho_f = rho_t - 1 - sum (2 eps - 2 pi eps^2) (Eq. rhofratiorhot);
rho_f is measured from the variance of beta F~ over independent runs (Eq. rhof)
with the error bar of Eq. (gaussian_err)."""
import numpy as np
import pytest

from paper_1711_02146_gb300.workloads import Workload, linear_betas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drivers():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02146_gb300 import build
    build.build()
    from paper_1711_02146_gb300 import drivers as d
    return d


def test_rho_f_and_rho_t_in_the_equilibrated_regime(drivers):
    w = Workload("hot", L=6, R=4000, disorder_seed=7, run_seed=0, betas=linear_betas(41, 0.25), n_sweeps=10)
    r = drivers.free_energy_variance(w, M=48, first_run_seed=100)
    t = len(w.betas) - 1
    assert r["eps"][1:].min() > 0
    # Eq. (rhotb): rho_t - 1 = 2 sum eps (rho_t from one run, averaged over the runs)
    assert abs((r["rho_t"][t] - 1) - (r["rho_t_grow"][t] - 1)) < 0.1 * (r["rho_t_grow"][t] - 1) + 4 * r["rho_t_err"][t]
    # Eq. (rhofgrow): rho_f = 2 pi sum eps^2, within the error of a variance over M runs
    assert abs(r["rho_f"][t] - r["rho_f_grow"][t]) < 3 * r["rho_f_err"][t]
    # Eq. (rhofratiorhot): the estimate from rho_t agrees with the measured rho_f
    assert abs(r["rho_f"][t] - r["rho_f_from_rho_t"][t]) < 3 * r["rho_f_err"][t] + 0.1 * r["rho_t"][t]


def test_hardness_adaptive_population(drivers):
    w = Workload("hard", L=6, R=200, disorder_seed=11, run_seed=3, betas=linear_betas(21, 3.0), n_sweeps=5)
    res = drivers.hardness_adaptive_population(w, R0=200, max_rounds=4)
    hist = res["history"]
    assert hist[0][0] == 200
    for (R_prev, rt_prev), (R_next, _) in zip(hist, hist[1:]):
        assert R_prev <= 100 * rt_prev                 # reran only when not equilibrated
        assert R_next == int(np.ceil(150 * rt_prev))   # with R = 150 rho_t
    if res["equilibrated"]:
        assert res["R"] > 100 * res["rho_t"]


def test_optimized_schedule_beats_constant_steps(drivers):
    # §V.A on a few L = 6 samples: equal sweeps per replica, smaller rho_t with the
    # constant-culling beta schedule and the 3/22/1 sweep schedule
    r = drivers.schedule_comparison(6, 4000, range(1, 13))
    assert abs(r["sweeps_opt"] - r["sweeps_unopt"]) <= 0.03 * r["sweeps_unopt"]
    assert r["n_steps_opt"] > 10
    assert r["geo_mean_ratio"] > 1.0


def test_katzgraber_young_vanishes_in_equilibrium(drivers):
    # Gaussian couplings, high temperatures, well-equilibrated populations:
    # the disorder average [e_l - e] is zero within its error (Eq. KY)
    r = drivers.katzgraber_young(4, 3000, range(1, 25), np.linspace(0.0, 1.2, 13), n_sweeps=5)
    for t in range(1, 13):
        assert abs(r["delta_KY"][t]) < 4 * r["delta_KY_err"][t] + 0.01, (t, r["delta_KY"][t], r["delta_KY_err"][t])
    assert r["e"][12] < r["e"][1] < 0
