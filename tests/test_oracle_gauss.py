"""Pins of the Gaussian-coupling oracle (the paper's model, §II.A) against facts
that do not come from the oracle itself: the normal law of the couplings, exact
enumeration of all states at L = 2 (partition function, energy, link overlap),
the Katzgraber-Young identity of Gaussian disorder (Eqs. KY, el), the Boltzmann
distribution reached by the Metropolis sweeps, and the closed forms behind the
acceptance thresholds and the resampling weights and sums."""
import itertools
import math

import numpy as np
import pytest

import oracle

SCALE = 2.0 ** -20


def _bonds(L):
    N = L ** 3

    def nb(n, d):
        x, y, z = n % L, (n // L) % L, n // (L * L)
        if d == 0:
            x = (x + 1) % L
        if d == 1:
            y = (y + 1) % L
        if d == 2:
            z = (z + 1) % L
        return x + L * (y + L * z)
    return [(n, nb(n, d), 3 * n + d) for n in range(N) for d in range(3)]


def _exact_l2(J, beta):
    """Exact ln Z, <E> and the bond correlations <s s>_b of an L = 2 sample."""
    L, N = 2, 8
    bonds = _bonds(L)
    states = np.array(list(itertools.product([1, -1], repeat=N)), dtype=np.int64)
    ss = np.stack([states[:, a] * states[:, b] for a, b, _ in bonds], axis=1)
    E = -(ss * np.array([J[k] for _, _, k in bonds], dtype=np.float64)).sum(axis=1)
    lw = -beta * E
    m = lw.max()
    w = np.exp(lw - m)
    Z = w.sum()
    p = w / Z
    return m + math.log(Z), float((p * E).sum()), (p[:, None] * ss).sum(axis=0), E, p


def test_couplings_are_standard_normal():
    J = np.concatenate([oracle.gcouplings(16, seed) for seed in (1, 2, 3)]).astype(np.float64) * SCALE
    n = J.size
    assert abs(J.mean()) < 4 / math.sqrt(n)
    assert abs(J.var() - 1.0) < 4 * math.sqrt(2.0 / n)
    # fourth moment of N(0,1) is 3; fraction beyond one sigma is 0.3173
    assert abs((J ** 4).mean() - 3.0) < 0.15
    assert abs((np.abs(J) > 1.0).mean() - 0.3173) < 0.01
    assert np.abs(J).max() <= 5.0
    Jq = oracle.gcouplings(8, 5)
    assert Jq.dtype == np.int32 and np.array_equal(Jq, oracle.gcouplings(8, 5))
    assert not np.array_equal(Jq, oracle.gcouplings(8, 6))


def test_energy_symmetries():
    L = 4
    Jq = oracle.gcouplings(L, 11)
    rng = np.random.default_rng(0)
    s = rng.choice([-1, 1], size=L ** 3).astype(np.int8)
    E = oracle.genergy(L, Jq, s)
    assert oracle.genergy(L, Jq, -s) == E                       # global flip
    assert oracle.genergy(L, Jq, np.ones(L ** 3, np.int8)) == -int(Jq.astype(np.int64).sum())
    # gauge: s -> g s, J_nm -> g_n g_m J_nm leaves E unchanged
    g = rng.choice([-1, 1], size=L ** 3)
    Jg = Jq.copy()
    for n, m, k in _bonds(L):
        Jg[k] = Jq[k] * g[n] * g[m]
    assert oracle.genergy(L, Jg, (s * g).astype(np.int8)) == E
    # a single flip changes E by 2 s_n h_n
    n0 = 13
    h = sum(int(Jq[k]) * int(s[m] if a == n0 else s[a]) for a, m, k in _bonds(L) if n0 in (a, m))
    s2 = s.copy()
    s2[n0] = -s2[n0]
    assert oracle.genergy(L, Jq, s2) - E == 2 * int(s[n0]) * h


@pytest.mark.parametrize("beta", [1e-6, 0.1, 0.7, 2.0])
def test_acceptance_threshold_is_the_boltzmann_factor(beta):
    """thr(dE) = floor(2^32 exp(-beta dE)), capped at 2^32 - 2, against the closed
    form in exact decimal arithmetic (60 digits): equal, or one below when 2^32 p
    lies within a few ulp above an integer."""
    import decimal
    decimal.getcontext().prec = 60
    rng = np.random.default_rng(1)
    dEs = [1, 2, 4095, 2 ** 20, 3 * 2 ** 20 + 17] + [int(x) for x in rng.integers(1, 40 * 2 ** 20, size=300)]
    prev = None
    for dE in sorted(dEs):
        exact = (decimal.Decimal(-beta) * decimal.Decimal(dE) / decimal.Decimal(2 ** 20)).exp() * (2 ** 32)
        want = min(int(exact), 2 ** 32 - 2)      # floor of a positive number
        thr = oracle.gacceptance_threshold(beta, dE)
        assert thr in (want, want - 1), (beta, dE, thr, want)
        if thr != want:
            assert exact - int(exact) < decimal.Decimal(2 ** 32) * decimal.Decimal(2) ** -50
        assert prev is None or thr <= prev     # monotone in dE
        prev = thr
    if beta < 1e-4:
        assert oracle.gacceptance_threshold(beta, 1) == 2 ** 32 - 2   # the cap: "always" stays ΔE <= 0 only


def test_reweighting_is_eqs_tau_q_and_eq_num_elim():
    """The resampling quantities of a population with real energies against the
    paper's definitions computed independently: each weight against the exact
    exponential (60-digit decimal), S' against the correctly rounded sum of exact
    weights (math.fsum) within the n-ulp bound of a sum of positive terms,
    sum_i tau_i = R, tau ratios = Boltzmann ratios, the culling fraction against
    Eq. (eq_num_elim) summed exactly, and shift invariance (weights measured from
    E_min)."""
    import decimal
    decimal.getcontext().prec = 60
    rng = np.random.default_rng(2)
    u = 2.0 ** -53
    for dbeta in (0.013, 0.2, 1.5):
        for d in [0, 1, 4095, 4096, 2 ** 24 - 1, 2 ** 24, 3 * 2 ** 30] + [int(v) for v in rng.integers(0, 2 ** 36, 50)]:
            exact = float((decimal.Decimal(-dbeta) * decimal.Decimal(d) / decimal.Decimal(2 ** 20)).exp())
            x = dbeta * d * SCALE
            # one rounding of the argument (relative u, so absolute u x) and one of exp
            assert abs(oracle.gweight(dbeta, d) - exact) <= (2 * u + 2 * u * x) * exact + 1e-300
    for n, R, dbeta in ((1, 1, 0.5), (700, 1000, 0.3), (5000, 4000, 0.05), (20000, 20000, 1.1)):
        E = rng.normal(-1.5 * 1000, 40.0, n)
        Eq = np.rint(E / SCALE).astype(np.int64)
        Emin, S, eps, tau = oracle.greweight(Eq, R, dbeta)
        assert Emin == int(Eq.min())
        w = [float((decimal.Decimal(-dbeta) * decimal.Decimal(int(e - Emin)) / decimal.Decimal(2 ** 20)).exp())
             for e in Eq]
        S_exact = math.fsum(w)
        assert abs(S - S_exact) <= (n + 2) * u * S_exact
        assert abs(math.fsum(tau) - R) <= 1e-12 * R
        i, j = rng.integers(0, n, 2)
        ratio = math.exp(-dbeta * (int(Eq[i]) - int(Eq[j])) * SCALE)
        assert abs(tau[i] / tau[j] - ratio) <= 1e-12 * ratio
        eps_exact = math.fsum(max(0.0, 1.0 - R * wk / S_exact) for wk in w) / R
        assert abs(eps - eps_exact) <= 1e-12 * max(eps_exact, 1e-300) + 1e-15
        # the same population shifted by a constant energy: the same S', tau and eps
        E2, S2, eps2, tau2 = oracle.greweight(Eq + 123456789, R, dbeta)
        assert E2 == Emin + 123456789 and S2 == S and eps2 == eps and np.array_equal(tau2, tau)
    with pytest.raises(RuntimeError):
        oracle.greweight(np.zeros(0, np.int64), 10, 0.1)


def test_culling_fraction_of_gaussian_energies_is_eq_eps():
    """Eq. (eps): for normally distributed energies and small dbeta sigma, the
    expected culling fraction is dbeta sigma_E / sqrt(2 pi) to leading order."""
    rng = np.random.default_rng(5)
    n, sigma = 200_000, 30.0
    Eq = np.rint(rng.normal(-1200.0, sigma, n) / SCALE).astype(np.int64)
    for x in (0.005, 0.02):
        dbeta = x / sigma
        _, _, eps, _ = oracle.greweight(Eq, n, dbeta)
        want = x / math.sqrt(2 * math.pi)
        assert abs(eps - want) < 0.03 * want + 4 / math.sqrt(n) * want, (x, eps, want)


def test_katzgraber_young_identity_by_enumeration():
    """For Gaussian disorder [<E>/N] = -beta (N_b/N)(1 - [<q_l>]) exactly (Eqs. KY, el);
    it holds for the oracle's couplings over many L = 2 samples within the error."""
    beta, d = 1.1, []
    bonds = _bonds(2)
    for seed in range(1, 801):
        J = oracle.gcouplings(2, seed).astype(np.float64) * SCALE
        _, Em, corr, _, _ = _exact_l2(J, beta)
        ql = float((corr ** 2).mean())
        d.append(-3 * beta * (1 - ql) - Em / 8)
    d = np.array(d)
    assert abs(d.mean()) < 3.5 * d.std() / math.sqrt(d.size)
    # and a biased coupling law would break it: shift every J by +0.5
    d2 = []
    for seed in range(1, 401):
        J = oracle.gcouplings(2, seed).astype(np.float64) * SCALE + 0.5
        _, Em, corr, _, _ = _exact_l2(J, beta)
        d2.append(-3 * beta * (1 - float((corr ** 2).mean())) - Em / 8)
    d2 = np.array(d2)
    assert abs(d2.mean()) > 5 * d2.std() / math.sqrt(d2.size)


@pytest.mark.parametrize("L", [4, 6])
def test_sweep_energy_changes_add_up(L):
    """The energy change a sweep reports equals the energy recomputed from scratch
    (every flip's dE uses the right six bonds; at L = 2 the x+1 and x-1 bonds
    join the same pair, so this needs L >= 4)."""
    Jq = oracle.gcouplings(L, 31 + L)
    rng = np.random.default_rng(L)
    for j, beta in enumerate((0.2, 0.9, 3.0)):
        s = rng.choice([-1, 1], size=L ** 3).astype(np.int8)
        s2, dE = oracle.gsweep_replica(L, Jq, s, 5, 0, j, 2, 3, beta)
        assert oracle.genergy(L, Jq, s2) - oracle.genergy(L, Jq, s) == dE
        assert (s2 != s).any()


def test_metropolis_uniform_is_uniform_and_slots_are_independent():
    """The Gaussian model's Metropolis uniform (a random-stream convention: its upper
    16 bits from one Philox stream, its lower 16 bits from a second).  Over 2^15 slots
    of one site and half-sweep it accepts a flip of threshold p 2^32 at rate p
    (binomial bound) and its nibbles are uniform (chi-square); neighbouring slots
    share an upper or a lower half no more often than chance allows, and so do the two
    halves of one uniform (a wrong half, word or counter would make them equal); other
    half-sweeps, sites, steps, populations and seeds draw other uniforms."""
    n = 1 << 15
    U = np.array([oracle.gmetropolis_uniform(7, 0, 5, 1, 0, j, 3) for j in range(n)], dtype=np.uint64)
    for p in (0.5, 0.25, 0.01):
        rate = float((U < int(p * 2 ** 32)).mean())
        assert abs(rate - p) < 5 * math.sqrt(p * (1 - p) / n)
    hi, lo = U >> np.uint64(16), U & np.uint64(0xFFFF)
    for d in (1, 2, 3, 4, 8):   # slots of one word, one block, one group
        assert (hi[d:] == hi[:-d]).sum() < 8 and (lo[d:] == lo[:-d]).sum() < 8
    assert (hi == lo).sum() < 8
    for v in (hi >> np.uint64(12), lo >> np.uint64(12), hi & np.uint64(15), lo & np.uint64(15)):
        c = np.bincount(v.astype(np.int64), minlength=16)
        chi2 = float(((c - n / 16) ** 2 / (n / 16)).sum())
        assert chi2 < 15 + 5 * math.sqrt(30)
    for seed, pop, site, sweep, colour, t in ((7, 0, 5, 1, 1, 3), (7, 0, 6, 1, 0, 3), (7, 0, 5, 2, 0, 3),
                                              (7, 0, 5, 1, 0, 4), (7, 1, 5, 1, 0, 3), (8, 0, 5, 1, 0, 3)):
        V = np.array([oracle.gmetropolis_uniform(seed, pop, site, sweep, colour, j, t) for j in range(256)],
                     dtype=np.uint64)
        assert (V == U[:256]).sum() < 2


def test_sweeps_sample_the_boltzmann_distribution():
    L, beta, seed = 2, 0.8, 21
    Jq = oracle.gcouplings(L, seed)
    _, _, _, E, p = _exact_l2(Jq.astype(np.float64) * SCALE, beta)
    Eq = np.rint(E / SCALE).astype(np.int64)
    levels, inv = np.unique(Eq, return_inverse=True)
    pl = np.bincount(inv, weights=p)
    rng = np.random.default_rng(3)
    n_chains, counts = 4000, np.zeros(levels.size)
    for j in range(n_chains):
        s = rng.choice([-1, 1], size=8).astype(np.int8)
        s, _ = oracle.gsweep_replica(L, Jq, s, 99, 0, j, 1, 30, beta)
        counts[np.searchsorted(levels, oracle.genergy(L, Jq, s))] += 1
    exp_ = pl * n_chains
    keep = exp_ > 5
    chi2 = (((counts[keep] - exp_[keep]) ** 2) / exp_[keep]).sum()
    dof = keep.sum() - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def test_run_reproduces_exact_free_energy_energy_and_link_overlap():
    L, seed, R = 2, 7, 30000
    betas = np.linspace(0.0, 1.5, 16)
    run = oracle.GRun(oracle.RunConfig(L=L, R=R, disorder_seed=seed, run_seed=3, betas=betas, n_sweeps=4, n_pop=2))
    run.run()
    J = run.couplings().astype(np.float64) * SCALE
    for t in (5, 10, 15):
        lnZ, Em, corr, _, _ = _exact_l2(J, betas[t])
        o0, o1 = run.obs(t, 0), run.obs(t, 1)
        assert abs(o0["minus_beta_F"] - lnZ) < 0.01
        assert abs(o1["minus_beta_F"] - lnZ) < 0.01
        assert abs(o0["mean_E"] - Em) < 0.05
        ql_exact = float((corr ** 2).mean())
        assert abs(o0["ql_mean"] - ql_exact) < 0.01
        assert o0["ql_mean"] == o1["ql_mean"] and o0["q_pairs"] == min(o0["R_tilde"], o1["R_tilde"])
        assert abs(o0["delta_KY"] - (-3 * betas[t] * (1 - o0["ql_mean"]) - o0["mean_E"] / 8)) < 1e-12
    # population and histograms are consistent with the observables
    s, lab, E = run.population(0)
    o = run.obs(run.t, 0)
    assert s.shape[0] == o["R_tilde"] and int(E.sum()) == o["sum_E"] and int(E.min()) == o["E_min"]
    assert all(oracle.genergy(L, run.couplings(), s[j]) == E[j] for j in range(0, s.shape[0], 997))
    assert run.q_hist(run.t).sum() == o["q_pairs"] and run.q_hist(run.t, link=True).sum() == o["q_pairs"]


def test_run_is_independent_of_thread_count():
    betas = np.linspace(0, 2.0, 6)
    outs = []
    for threads in (1, 3):
        r = oracle.GRun(oracle.RunConfig(L=4, R=700, disorder_seed=2, run_seed=8, betas=betas, n_sweeps=2,
                                         n_threads=threads))
        r.run()
        outs.append((r.population(0), r.obs(r.t, 0)))
    (a, oa), (b, ob) = outs
    assert all(np.array_equal(x, y) for x, y in zip(a, b)) and oa == ob


def test_adaptive_schedule_holds_the_culling_fraction():
    """§IV.B with Gaussian couplings: every step but the last has the largest dbeta
    whose expected culling fraction does not exceed the target; the run ends at
    beta_max; the free energy still follows the exact one (L = 2)."""
    eps, bmax = 0.25, 2.0
    run = oracle.GRun(oracle.RunConfig(L=2, R=20000, disorder_seed=5, run_seed=6, betas=None, n_temps=400,
                                       beta_max=bmax, eps_target=eps, n_sweeps=3))
    run.run()
    T = run.t
    betas = [run.obs(t)["beta"] for t in range(T + 1)]
    assert betas[-1] == bmax and all(b2 > b1 for b1, b2 in zip(betas, betas[1:]))
    for t in range(1, T + 1):
        e = run.obs(t)["eps_expected"]
        assert e <= eps
        if t < T:
            assert e >= eps * (1 - 1e-9)
    J = run.couplings().astype(np.float64) * SCALE
    for t in (T // 2, T):
        lnZ, _, _, _, _ = _exact_l2(J, betas[t])
        assert abs(run.obs(t)["minus_beta_F"] - lnZ) < 0.02
