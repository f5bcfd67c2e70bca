"""GPU parity of the Gaussian-coupling model (§II.A) against the oracle: couplings,
spins, labels, energies, copy numbers, overlap and link-overlap histograms and
every integer observable bit for bit; FP64 observables to 1e-12 relative.

The oracle computes the resampling as Eqs. (tau), (Q) and (eq_num_elim) define it
(one exponential per replica, plain sums in slot order); the GPU computes the same
quantities in its own arithmetic (table products, tree sums), so tau agrees to the
1e-12 tolerance rather than to the bit.  A copy number is then fixed by both sides
unless the replica's uniform word falls in the band of thresholds that tau's
tolerance spans; every step counts the replicas in that band (expected number about
R * 1e-12 * 2: none in practice), and all other copy numbers must agree exactly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 1e-12
INT_OBS = ("t", "R_tilde", "sum_E", "E_min", "E_min_prev", "culled", "sum_eta2", "n_families", "E0", "q_pairs",
           "q_abs_le_02", "ql_sum")
FLOAT_OBS = ("beta", "dbeta", "sum_E2", "mean_E", "var_E", "S_prime", "lnQ", "minus_beta_F", "eps_expected", "rho_t",
             "S_f", "rho_s", "g0_tilde", "g0_bar", "I02", "ql_mean", "e_l", "delta_KY")


@pytest.fixture(scope="module")
def pa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02146_gb300 import build, pa as pa_mod
    build.build()
    return pa_mod


def make_pair(pa, oracle_lib, L, R, betas, n_sweeps, n_pop=1, seed=1, run_seed=2):
    gpu = pa.Run(L, R, seed, run_seed, betas, n_sweeps=n_sweeps, n_pop=n_pop, model=pa.PA_MODEL_GAUSS)
    ref = oracle_lib.GRun(oracle_lib.RunConfig(L=L, R=R, disorder_seed=seed, run_seed=run_seed, betas=betas,
                                               n_sweeps=n_sweeps, n_pop=n_pop))
    return gpu, ref


def band_slots(oracle_lib, E_old, R, dbeta, run_seed, pop, t, rel=REL):
    """Old slots whose copy number is not fixed by tau to relative precision rel: the
    nearest-integer rule is monotone in tau, so a slot is in the band when the
    oracle's rule gives different copy numbers at tau (1 - rel) and tau (1 + rel)."""
    _, _, _, tau = oracle_lib.greweight(E_old, R, dbeta)
    lo = oracle_lib.resample_tau(tau * (1.0 - rel), run_seed, t, pop)
    hi = oracle_lib.resample_tau(tau * (1.0 + rel), run_seed, t, pop)
    return np.nonzero(lo != hi)[0]


def assert_counts(gpu, ref, oracle_lib, E_old, R, dbeta, run_seed, t, pop=0):
    band = band_slots(oracle_lib, E_old, R, dbeta, run_seed, pop, t)
    assert band.size == 0, f"t={t} pop {pop}: {band.size} replicas in the tolerance band {band[:5]}"
    assert np.array_equal(gpu.copy_counts(pop), ref.last_counts(pop)), f"copy numbers at t={t} pop {pop}"


def obs_scale(o, k):
    """Magnitude that bounds the rounding of observable k: its own, except for
    Delta_KY = e_l - <E>/N (the Katzgraber-Young check), a difference of two O(1)
    terms that nearly cancel, whose rounding is relative to those terms."""
    if k == "delta_KY":
        return abs(o["e_l"]) + abs(o["e_l"] - o["delta_KY"])
    return abs(o[k])


def assert_obs(g, r, ctx):
    for k in INT_OBS:
        assert g[k] == r[k], f"{ctx} {k}: gpu {g[k]} oracle {r[k]}"
    for k in FLOAT_OBS:
        a, b = g[k], r[k]
        if a == b:
            continue
        scale = max(obs_scale(g, k), obs_scale(r, k))
        assert abs(a - b) <= REL * scale + 1e-300, f"{ctx} {k}: gpu {a!r} oracle {b!r}"


def assert_state(gpu, ref, n_pop, ctx):
    for p in range(n_pop):
        s, lab, E = gpu.population(p)
        rs, rlab, rE = ref.population(p)
        assert s.shape == rs.shape, f"{ctx} pop {p}: size {s.shape[0]} vs {rs.shape[0]}"
        assert np.array_equal(lab, rlab), f"{ctx} pop {p}: labels"
        assert np.array_equal(E, rE), f"{ctx} pop {p}: energies"
        bad = np.nonzero(np.any(s != rs, axis=1))[0]
        assert bad.size == 0, f"{ctx} pop {p}: {bad.size} replicas differ, first {bad[:5]}"


@pytest.mark.parametrize("L,R", [(2, 77), (4, 700), (6, 555), (8, 1333), (10, 515), (12, 300), (14, 129), (16, 65)])
def test_stepwise(pa, oracle_lib, L, R):
    betas = np.linspace(0.0, 2.5, 5)
    gpu, ref = make_pair(pa, oracle_lib, L, R, betas, 2, seed=L, run_seed=50 + R)
    assert np.array_equal(gpu.gcouplings(), ref.couplings())
    assert_state(gpu, ref, 1, "t=0")
    assert_obs(gpu.gobs(0), ref.obs(0), "t=0")
    for t in range(1, len(betas)):
        E_old = ref.population(0)[2]
        assert gpu.step() == 0
        ref.step()
        assert_counts(gpu, ref, oracle_lib, E_old, R, betas[t] - betas[t - 1], 50 + R, t)
        assert_state(gpu, ref, 1, f"t={t}")
        assert_obs(gpu.gobs(t), ref.obs(t), f"t={t}")
    assert gpu.step() == pa.PA_DONE


def test_two_populations_overlaps(pa, oracle_lib):
    betas = np.linspace(0.0, 3.0, 9)
    gpu, ref = make_pair(pa, oracle_lib, 6, 900, betas, 3, n_pop=2, seed=3, run_seed=4)
    for t in range(len(betas)):
        if t:
            gpu.step()
            ref.step()
        for p in range(2):
            assert_obs(gpu.gobs(t, p), ref.obs(t, p), f"t={t} pop {p}")
        assert np.array_equal(gpu.q_hist(t), ref.q_hist(t)), f"q histogram at t={t}"
        assert np.array_equal(gpu.ql_hist(t), ref.q_hist(t, link=True)), f"q_l histogram at t={t}"
    assert_state(gpu, ref, 2, "end")


def test_longer_run_and_sweep_schedule(pa, oracle_lib):
    betas = np.linspace(0.0, 3.0, 21)
    sweeps = np.array([0] + [3] * 6 + [7] * 8 + [1] * 6, dtype=np.int32)
    gpu = pa.Run(8, 3000, 9, 10, betas, sweeps_per_step=sweeps, model=pa.PA_MODEL_GAUSS)
    ref = oracle_lib.GRun(oracle_lib.RunConfig(L=8, R=3000, disorder_seed=9, run_seed=10, betas=betas,
                                               sweeps_per_step=sweeps))
    gpu.run()
    ref.run()
    for t in (1, 10, 20):
        assert_obs(gpu.gobs(t), ref.obs(t), f"t={t}")
    assert_state(gpu, ref, 1, "end")


def test_gaussian_runs_refuse_the_pm1_readers(pa):
    run = pa.Run(4, 100, 1, 1, np.linspace(0, 1, 3), model=pa.PA_MODEL_GAUSS)
    for call in (lambda: run.obs(0), lambda: run.energy_hist(0), lambda: run.replicas(0, 0, 5)):
        with pytest.raises(pa.PAError) as e:
            call()
        assert e.value.status == pa.PA_ERR_INVALID
    pm1 = pa.Run(4, 100, 1, 1, np.linspace(0, 1, 3))
    with pytest.raises(pa.PAError):
        pm1.gobs(0)


def test_full_size_sampled_steps(pa, oracle_lib):
    """L = 10, R = 1e6 with Gaussian couplings (the benchmark's Gaussian workload),
    two steps in the benchmark's launch configuration: the resampling is recomputed
    from the GPU's energies with the oracle's definitions (weights, S', culling sum,
    every copy number), and sampled replicas are swept again by the oracle from their
    parents."""
    import bench
    w = bench.gaussian_workload()
    gpu = pa.Run.from_workload(w)
    L, N, R = w.L, w.N, w.R
    Jq = gpu.gcouplings()
    assert np.array_equal(Jq, oracle_lib.gcouplings(L, w.disorder_seed))
    rng = np.random.default_rng(0)
    for _ in range(2):
        s_old, lab_old, E_old = gpu.population()
        for j in rng.integers(0, len(E_old), 16):
            assert oracle_lib.genergy(L, Jq, s_old[j]) == E_old[j]
        gpu.step()
        t = gpu.t
        o = gpu.gobs(t)
        # resampling, from the oracle's definitions (Eqs. tau, Q, eq_num_elim) on the GPU's energies
        Emin, S, eps, tau = oracle_lib.greweight(E_old, R, o["dbeta"])
        assert o["E_min_prev"] == Emin
        assert abs(o["S_prime"] - S) <= REL * S, (o["S_prime"], S)
        assert abs(o["eps_expected"] - eps) <= REL * eps, (o["eps_expected"], eps)
        lnQ = np.log(S / len(E_old)) - o["dbeta"] * Emin * 2.0 ** -20
        assert abs(o["lnQ"] - lnQ) <= REL * (abs(lnQ) + abs(o["dbeta"] * Emin * 2.0 ** -20))
        counts = gpu.copy_counts()
        assert counts.size == len(E_old)
        want = oracle_lib.resample_tau(tau, w.run_seed, t)
        lo = oracle_lib.resample_tau(tau * (1.0 - REL), w.run_seed, t)
        hi = oracle_lib.resample_tau(tau * (1.0 + REL), w.run_seed, t)
        band = np.nonzero(lo != hi)[0]
        assert band.size <= 2, f"{band.size} replicas in the tolerance band"
        fixed = np.setdiff1d(np.arange(len(E_old)), band)
        assert np.array_equal(counts[fixed], want[fixed])
        assert np.all((counts[band] == lo[band]) | (counts[band] == hi[band]))
        parents = gpu.parents()
        assert parents.size == counts.sum() == o["R_tilde"]
        assert np.array_equal(parents, np.repeat(np.arange(len(E_old), dtype=np.int32), counts))
        s_new, lab_new, E_new = gpu.population()
        assert np.array_equal(lab_new, lab_old[parents])
        for j in rng.integers(0, len(E_new), 24):
            ref, dE = oracle_lib.gsweep_replica(L, Jq, s_old[parents[j]], w.run_seed, 0, int(j), t, w.n_sweeps,
                                                gpu.beta(t))
            assert np.array_equal(s_new[j], ref), f"slot {j}"
            assert E_new[j] == E_old[parents[j]] + dE
        # exact moments of the new population
        assert o["sum_E"] == int(E_new.sum()) and o["E_min"] == int(E_new.min())
        assert o["sum_E2"] == float(sum(int(e) * int(e) for e in E_new.tolist()))


@pytest.mark.parametrize("L,R,eps,bmax,n_pop", [(4, 900, 0.3, 2.5, 1), (6, 1500, 0.2, 3.0, 2), (10, 4000, 0.45, 2.0, 1)])
def test_adaptive_schedule(pa, oracle_lib, L, R, eps, bmax, n_pop):
    """§IV.B with Gaussian couplings: the GPU bisects on its own culling fractions, the
    oracle on the definition's; the two agree to the tolerance, so the chosen
    temperatures agree to it too (the bisection's last halvings may split the
    difference), and with them every population and observable."""
    gpu = pa.Run(L, R, 3, 40 + L, None, n_temps=400, beta_max=bmax, eps_target=eps, n_sweeps=2, n_pop=n_pop,
                 model=pa.PA_MODEL_GAUSS)
    ref = oracle_lib.GRun(oracle_lib.RunConfig(L=L, R=R, disorder_seed=3, run_seed=40 + L, betas=None, n_temps=400,
                                               beta_max=bmax, eps_target=eps, n_sweeps=2, n_pop=n_pop))
    t = 0
    while True:
        E_old = [ref.population(p)[2] for p in range(n_pop)]
        rg, rr = gpu.step(), ref.step()
        if rr == oracle_lib.DONE:
            assert rg == pa.PA_DONE
            break
        assert rg == 0
        t += 1
        for p in range(n_pop):
            assert_obs(gpu.gobs(t, p), ref.obs(t, p), f"t={t} pop {p}")
            assert_counts(gpu, ref, oracle_lib, E_old[p], R, ref.obs(t)["dbeta"], 40 + L, t, p)
        assert_state(gpu, ref, n_pop, f"t={t}")
    assert t >= 3 and gpu.gobs(t)["beta"] == bmax
    assert all(gpu.gobs(u)["eps_expected"] <= eps for u in range(1, t + 1))


@pytest.mark.parametrize("L,R,eps,bmax", [(6, 1500, 0.2, 3.0), (10, 300_000, 0.272, 1.0)])
def test_adaptive_bisection_one_launch_equals_launch_per_halving(pa, L, R, eps, bmax):
    """§IV.B: the bisection's halvings in one cooperative launch take the decisions of
    the launch-per-halving form from the same sums, so every temperature, population
    and observable of the two runs is the same to the bit (R = 3e5 spans 1172 chunk
    sums: two levels of the fixed-order tree and several chunks per block)."""
    runs = []
    for one_launch in (1, 0):
        r = pa.Run(L, R, 5, 70 + L, None, n_temps=400, beta_max=bmax, eps_target=eps, n_sweeps=1,
                   model=pa.PA_MODEL_GAUSS)
        assert pa.lib().pa_debug_bisect(r._h, one_launch, -1) == pa.PA_OK
        runs.append(r)
    assert pa.lib().pa_debug_bisect(runs[0]._h, 2, -1) == pa.PA_ERR_INVALID
    assert pa.lib().pa_debug_bisect(runs[0]._h, 0, 3) == pa.PA_ERR_INVALID
    assert pa.lib().pa_debug_bisect(runs[0]._h, 1, -2) == pa.PA_ERR_INVALID
    t = 0
    while True:
        a, b = runs[0].step(), runs[1].step()
        assert a == b
        if a == pa.PA_DONE:
            break
        t += 1
        oa, ob = runs[0].gobs(t), runs[1].gobs(t)
        for k in INT_OBS + FLOAT_OBS:
            va, vb = oa[k], ob[k]
            assert va == vb or (va != va and vb != vb), (t, k, va, vb)
        assert oa["eps_expected"] <= eps
    assert t >= 3 and runs[0].gobs(t)["beta"] == bmax
    for p in (0, 1, 2):
        assert np.array_equal(runs[0].population()[p], runs[1].population()[p])
    linear = pa.Run(4, 100, 1, 2, np.linspace(0.0, 1.0, 5), n_sweeps=1, model=pa.PA_MODEL_GAUSS)
    pm1 = pa.Run(4, 100, 1, 2, None, n_temps=10, beta_max=1.0, eps_target=0.3, n_sweeps=1)
    assert pa.lib().pa_debug_bisect(linear._h, 1, -1) == pa.PA_ERR_INVALID
    assert pa.lib().pa_debug_bisect(pm1._h, 1, -1) == pa.PA_ERR_INVALID
    for r in runs + [linear, pm1]:
        r.close()
