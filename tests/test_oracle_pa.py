"""Pins for full oracle PA runs against exact results at L = 2 and L = 3.

  * Eq. (betaF): the mean of -beta_t F~ over independent runs matches the exact
    ln Z(beta_t) from enumeration within its statistical error at every step;
  * population averages <E>_t match the exact thermal average;
  * the lowest energy found reaches the exact ground state, and g~0 matches the
    exact ground-state weight (§II.A);
  * the culled count matches the expected culling fraction, Eq. (eq_num_elim);
  * the overlap histogram of two independent populations matches the exact P(q)
    from all pairs of states (§II.A);
  * family bookkeeping invariants and the adaptive schedule of §IV.B.
"""
import numpy as np
import pytest
from scipy import stats


def exact_lnZ_and_E(L, g, beta):
    N = L ** 3
    k = np.arange(3 * N + 1)
    E = (2 * k - 3 * N).astype(np.float64)
    m = g > 0
    x = np.log(g[m].astype(np.float64)) - beta * E[m]
    mx = x.max()
    w = np.exp(x - mx)
    lnZ = mx + np.log(w.sum())
    meanE = (w * E[m]).sum() / w.sum()
    return lnZ, meanE


@pytest.mark.parametrize("L,R,M,T,beta_max,S", [(2, 2000, 16, 21, 2.0, 5), (3, 3000, 10, 16, 1.5, 10)])
def test_free_energy_and_energy_match_enumeration(oracle_lib, L, R, M, T, beta_max, S):
    betas = np.array([t * beta_max / (T - 1) for t in range(T)])
    runs = []
    for m in range(M):
        run = oracle_lib.Run(oracle_lib.RunConfig(L=L, R=R, disorder_seed=21, run_seed=500 + m, betas=betas,
                                                  n_sweeps=S))
        run.run()
        runs.append(run)
    J = runs[0].couplings()
    g = oracle_lib.enumerate_levels(L, J)
    N = L ** 3
    for t in range(T):
        lnZ, meanE = exact_lnZ_and_E(L, g, betas[t])
        F = np.array([r.obs(t)["minus_beta_F"] for r in runs])
        E = np.array([r.obs(t)["mean_E"] for r in runs])
        if t == 0:
            assert np.all(F == N * np.log(2.0))
            continue
        se_F = F.std(ddof=1) / np.sqrt(M)
        se_E = E.std(ddof=1) / np.sqrt(M)
        assert abs(F.mean() - lnZ) < 4 * se_F + 2e-3, (t, F.mean(), lnZ, se_F)
        assert abs(E.mean() - meanE) < 4 * se_E + 2e-3, (t, E.mean(), meanE, se_E)


def test_ground_state_and_g0(oracle_lib):
    L, R = 3, 10000
    betas = np.array([t * 5.0 / 50 for t in range(51)])
    run = oracle_lib.Run(oracle_lib.RunConfig(L=L, R=R, disorder_seed=33, run_seed=7, betas=betas, n_sweeps=10))
    run.run()
    g = oracle_lib.enumerate_levels(L, run.couplings())
    N = L ** 3
    E0_exact = 2 * int(np.nonzero(g)[0][0]) - 3 * N
    assert run.obs(50)["E0"] == E0_exact
    for t in range(51):
        assert run.obs(t)["E0"] >= E0_exact
    # g~0 at an intermediate temperature against the exact ground-state weight
    t = 10
    o = run.obs(t)
    lnZ, _ = exact_lnZ_and_E(L, g, betas[t])
    k0 = (o["E0"] + 3 * N) // 2
    p_exact = np.exp(np.log(g[k0]) - betas[t] * o["E0"] - lnZ)
    se = np.sqrt(p_exact * (1 - p_exact) * o["rho_t"] / o["R_tilde"])
    assert abs(o["g0_tilde"] - p_exact) < 5 * se + 1e-3
    # Eq. (g0) with the exact E0 and F~: g0_bar = 2 exp(-beta E0 - (-beta F~))
    assert o["g0_bar"] == pytest.approx(2 * np.exp(-betas[t] * o["E0"] - o["minus_beta_F"]), rel=1e-12)


def test_culling_matches_expected_fraction(oracle_lib):
    betas = np.array([t * 3.0 / 40 for t in range(41)])
    run = oracle_lib.Run(oracle_lib.RunConfig(L=4, R=5000, disorder_seed=4, run_seed=9, betas=betas, n_sweeps=5))
    run.run()
    culled = sum(run.obs(t)["culled"] for t in range(1, 41))
    expected = sum(run.obs(t)["eps_expected"] * 5000 for t in range(1, 41))
    assert abs(culled - expected) < 5 * np.sqrt(expected) + 5
    for t in range(41):
        o = run.obs(t)
        assert abs(o["R_tilde"] - 5000) < 10 * np.sqrt(5000)


def test_initial_step_and_family_invariants(oracle_lib):
    betas = np.array([t * 2.0 / 20 for t in range(21)])
    R = 3000
    run = oracle_lib.Run(oracle_lib.RunConfig(L=4, R=R, disorder_seed=8, run_seed=2, betas=betas, n_sweeps=3))
    o = run.obs(0)
    assert o["R_tilde"] == R and o["n_families"] == R and o["sum_eta2"] == R
    assert o["rho_t"] == 1.0
    assert o["rho_s"] == pytest.approx(1.0, rel=1e-12)
    assert o["minus_beta_F"] == 64 * np.log(2.0)
    for _ in range(12):
        run.step()
    eta, m = run.family_hist()
    o = run.obs(run.t)
    assert (eta * m).sum() == o["R_tilde"]
    assert m.sum() == o["n_families"]
    assert (eta * eta * m).sum() == o["sum_eta2"]
    nu = eta / o["R_tilde"]
    assert o["S_f"] == pytest.approx(-(m * nu * np.log(nu)).sum(), rel=1e-12)
    s, lab, E = run.population()
    assert np.all(np.diff(lab) >= 0)            # labels stay sorted along slots
    counts = run.last_counts()
    assert counts.sum() == o["R_tilde"]
    assert (counts == 0).sum() == o["culled"]


def test_overlap_histogram_matches_exact_pairs(oracle_lib):
    L, R, beta = 2, 30000, 0.7
    N = L ** 3
    run = oracle_lib.Run(oracle_lib.RunConfig(L=L, R=R, disorder_seed=12, run_seed=3, betas=np.array([0.0, beta]),
                                              n_sweeps=0, sweeps_per_step=np.array([0, 100], dtype=np.int32),
                                              n_pop=2, q_bins=65))
    run.run()
    J = run.couplings()
    states = np.array([[1 if (i >> n) & 1 == 0 else -1 for n in range(N)] for i in range(2 ** N)], dtype=np.int8)
    E = np.array([oracle_lib.energy(L, J, s) for s in states], dtype=np.float64)
    w = np.exp(-beta * (E - E.min()))
    w /= w.sum()
    Q = states.astype(np.int64) @ states.astype(np.int64).T
    bins = ((Q + N) * 64 + N) // (2 * N)
    p = np.zeros(65)
    np.add.at(p, bins.ravel(), np.outer(w, w).ravel())
    h = run.q_hist(1)
    pairs = run.obs(1)["q_pairs"]
    assert h.sum() == pairs == min(run.obs(1, 0)["R_tilde"], run.obs(1, 1)["R_tilde"])
    keep = p * pairs >= 5
    assert h[~keep].sum() <= max(5, 5 * p[~keep].sum() * pairs)
    chi2 = ((h[keep] - pairs * p[keep]) ** 2 / (pairs * p[keep])).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-6
    # I(0.2): pairs with |q| <= 0.2
    small = sum(h[b] for b in range(65) if abs(-1 + 2 * b / 64) <= 0.2 + 1e-12)
    assert run.obs(1)["q_abs_le_02"] == small


def test_adaptive_schedule_holds_culling_fraction(oracle_lib):
    eps = 0.15
    run = oracle_lib.Run(oracle_lib.RunConfig(L=4, R=4000, disorder_seed=5, run_seed=6, n_temps=400, beta_max=3.0,
                                              eps_target=eps, n_sweeps=5))
    run.run()
    T = run.t
    betas = [run.beta(t) for t in range(T + 1)]
    assert betas[-1] == 3.0
    assert all(b2 > b1 for b1, b2 in zip(betas, betas[1:]))
    for t in range(1, T + 1):
        o = run.obs(t)
        assert o["eps_expected"] <= eps
        if t < T:
            assert o["eps_expected"] > eps * (1 - 1e-9)
        assert o["dbeta"] == pytest.approx(betas[t] - betas[t - 1], rel=1e-12, abs=1e-15)
    # Eq. (cullbeta) estimate of the first step: dbeta ~ eps sqrt(2 pi) / sigma_E
    sigma0 = np.sqrt(run.obs(0)["var_E"])
    assert betas[1] == pytest.approx(eps * np.sqrt(2 * np.pi) / sigma0, rel=0.2)


def test_results_independent_of_thread_count(oracle_lib):
    betas = np.array([t * 2.0 / 10 for t in range(11)])
    out = []
    for threads in (1, 3):
        run = oracle_lib.Run(oracle_lib.RunConfig(L=4, R=777, disorder_seed=1, run_seed=5, betas=betas, n_sweeps=4,
                                                  n_pop=2, n_threads=threads))
        run.run()
        out.append((run.population(0), run.population(1), run.q_hist(10), run.obs(10)))
    a, b = out
    for x, y in zip(a[0] + a[1], b[0] + b[1]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[2], b[2])
    assert a[3] == b[3]
