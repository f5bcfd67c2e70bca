"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer results — spins, labels, energies, copy numbers, population sizes,
energy/overlap/family histograms, the adaptive schedule — must match bit for
bit; FP64 observables to 1e-12 relative (the host-side estimators use the same
formulas on the same integer inputs, so in practice they match exactly except
the family entropy, whose device reduction order differs).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 1e-12
INT_OBS = ("t", "R_tilde", "sum_E", "sum_E2", "E_min", "kmin_prev", "culled", "sum_eta2", "n_families", "E0",
           "q_pairs", "q_abs_le_02")
FLOAT_OBS = ("beta", "dbeta", "mean_E", "var_E", "S_prime", "lnQ", "minus_beta_F", "eps_expected", "rho_t", "S_f",
             "rho_s", "g0_tilde", "g0_bar", "I02")


@pytest.fixture(scope="module")
def pa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02146_gb300 import build, pa as pa_mod
    build.build()
    return pa_mod


def make_pair(pa, oracle_lib, L, R, betas=None, **kw):
    gpu = pa.Run(L, R, kw.get("disorder_seed", 1), kw.get("run_seed", 2), betas,
                 n_temps=kw.get("n_temps", 0), beta_max=kw.get("beta_max", 0.0), eps_target=kw.get("eps_target", 0.0),
                 n_sweeps=kw.get("n_sweeps", 3), sweeps_per_step=kw.get("sweeps_per_step"), n_pop=kw.get("n_pop", 1),
                 q_bins=kw.get("q_bins", 65), R_cap=kw.get("R_cap", 0))
    ref = oracle_lib.Run(oracle_lib.RunConfig(L=L, R=R, disorder_seed=kw.get("disorder_seed", 1),
                                              run_seed=kw.get("run_seed", 2), betas=betas, n_temps=kw.get("n_temps", 0),
                                              beta_max=kw.get("beta_max", 0.0), eps_target=kw.get("eps_target", 0.0),
                                              n_sweeps=kw.get("n_sweeps", 3),
                                              sweeps_per_step=kw.get("sweeps_per_step"), n_pop=kw.get("n_pop", 1),
                                              q_bins=kw.get("q_bins", 65), R_cap=kw.get("R_cap", 0)))
    return gpu, ref


def assert_obs_equal(g, r, ctx=""):
    for k in INT_OBS:
        assert g[k] == r[k], f"{ctx} {k}: gpu {g[k]} oracle {r[k]}"
    for k in FLOAT_OBS:
        a, b = g[k], r[k]
        if a == b:          # includes equal infinities (e.g. g0_bar of a badly annealed run)
            continue
        assert abs(a - b) <= REL * max(abs(a), abs(b)) + 1e-300, f"{ctx} {k}: gpu {a!r} oracle {b!r}"


def assert_state_equal(gpu, ref, n_pop, ctx=""):
    for pop in range(n_pop):
        s, lab, E = gpu.population(pop)
        rs, rlab, rE = ref.population(pop)
        assert s.shape == rs.shape, f"{ctx} pop {pop}: population size {s.shape[0]} vs {rs.shape[0]}"
        assert np.array_equal(lab, rlab), f"{ctx} pop {pop}: labels"
        assert np.array_equal(E, rE), f"{ctx} pop {pop}: energies"
        bad = np.nonzero(np.any(s != rs, axis=1))[0]
        assert bad.size == 0, f"{ctx} pop {pop}: {bad.size} replicas differ, first {bad[:5]}"


def linear(T, bmax):
    return np.array([t * bmax / (T - 1) for t in range(T)])


@pytest.mark.parametrize("L,R,T,S", [(2, 37, 6, 3), (4, 1000, 8, 3), (4, 1, 5, 2), (6, 777, 5, 2), (8, 3333, 4, 2),
                                     (10, 515, 4, 2), (12, 300, 3, 1), (14, 129, 3, 1), (16, 65, 3, 1)])
def test_stepwise_bit_exact(pa, oracle_lib, L, R, T, S):
    betas = linear(T, 2.0)
    gpu, ref = make_pair(pa, oracle_lib, L, R, betas, n_sweeps=S, disorder_seed=L, run_seed=100 + R)
    assert np.array_equal(gpu.couplings(), ref.couplings())
    assert_state_equal(gpu, ref, 1, "t=0")
    assert_obs_equal(gpu.obs(0), ref.obs(0), "t=0")
    for t in range(1, T):
        assert gpu.step() == 0
        ref.step()
        assert np.array_equal(gpu.copy_counts(), ref.last_counts()), f"copy numbers at t={t}"
        assert_state_equal(gpu, ref, 1, f"t={t}")
        assert np.array_equal(gpu.energy_hist(t), ref.energy_hist(t)), f"energy histogram at t={t}"
        assert_obs_equal(gpu.obs(t), ref.obs(t), f"t={t}")
        eta, m = gpu.family_hist()
        reta, rm = ref.family_hist()
        assert np.array_equal(eta, reta) and np.array_equal(m, rm)
    assert gpu.step() == 1  # PA_DONE


@pytest.mark.parametrize("L,R", [(18, 61), (24, 40), (32, 21), (64, 8)])
def test_large_lattices_sweep_in_global_memory(pa, oracle_lib, L, R):
    """16 < L <= 64: the replica copy and the half-sweeps run in global memory, the
    reweighting keeps its level list in global memory; results are the oracle's."""
    betas = linear(3, 1.5)
    gpu, ref = make_pair(pa, oracle_lib, L, R, betas, n_sweeps=2, disorder_seed=L, run_seed=7 + R, n_pop=2)
    assert np.array_equal(gpu.couplings(), ref.couplings())
    for t in range(1, 3):
        assert gpu.step() == 0
        ref.step()
        assert np.array_equal(gpu.copy_counts(), ref.last_counts()), f"copy numbers at t={t}"
        assert_state_equal(gpu, ref, 2, f"t={t}")
        for p in range(2):
            assert np.array_equal(gpu.energy_hist(t, p), ref.energy_hist(t, p)), f"energy histogram at t={t}"
            assert_obs_equal(gpu.obs(t, p), ref.obs(t, p), f"t={t} pop {p}")
        assert np.array_equal(gpu.q_hist(t), ref.q_hist(t))
    with pytest.raises(pa.PAError):
        pa.sweep_shapes(L)


@pytest.mark.parametrize("L,R", [(4, 900), (10, 700), (18, 50)])
def test_extreme_temperatures(pa, oracle_lib, L, R):
    """Thresholds at both ends of the Metropolis test: beta ~ 1e-9 makes every
    threshold bit 1 for ~28 planes (long runs of the bitwise comparison), beta = 40
    makes every threshold 0 (no replica compares at all), and a jump between them
    culls hard.  Tile kernel (L <= 16) and global-memory kernel (L = 18)."""
    betas = np.array([0.0, 1e-9, 2e-9, 1e-6, 0.3, 1.0, 40.0, 40.0])
    gpu, ref = make_pair(pa, oracle_lib, L, R, betas, n_sweeps=2, run_seed=17 + L)
    for t in range(1, len(betas)):
        assert gpu.step() == 0
        ref.step()
        assert np.array_equal(gpu.copy_counts(), ref.last_counts()), f"copy numbers at t={t}"
        assert_state_equal(gpu, ref, 1, f"L={L} t={t}")
        assert_obs_equal(gpu.obs(t), ref.obs(t), f"L={L} t={t}")


def test_lattices_beyond_64_are_rejected(pa):
    for L in (66, 65, 17):
        with pytest.raises(pa.PAError) as e:
            pa.Run(L, 10, 1, 1, linear(3, 1.0))
        assert e.value.status == pa.PA_ERR_INVALID
    with pytest.raises(pa.PAError):   # Gaussian couplings stay within the shared-memory sweep
        pa.Run(18, 10, 1, 1, linear(3, 1.0), model=pa.PA_MODEL_GAUSS)


def test_c1_full_run(pa, oracle_lib):
    from paper_1711_02146_gb300.workloads import C1
    gpu = pa.Run.from_workload(C1)
    ref = oracle_lib.Run(oracle_lib.RunConfig(L=C1.L, R=C1.R, disorder_seed=C1.disorder_seed, run_seed=C1.run_seed,
                                              betas=C1.betas, n_sweeps=C1.n_sweeps))
    gpu.run()
    ref.run()
    assert_state_equal(gpu, ref, 1, "C1 end")
    for t in range(len(C1.betas)):
        assert np.array_equal(gpu.energy_hist(t), ref.energy_hist(t)), t
        assert_obs_equal(gpu.obs(t), ref.obs(t), f"C1 t={t}")


def test_two_populations_overlap(pa, oracle_lib):
    betas = linear(12, 3.0)
    gpu, ref = make_pair(pa, oracle_lib, 8, 2000, betas, n_sweeps=4, n_pop=2, disorder_seed=2, run_seed=9)
    gpu.run()
    ref.run()
    assert_state_equal(gpu, ref, 2, "two populations")
    for t in range(12):
        assert np.array_equal(gpu.q_hist(t), ref.q_hist(t)), t
        for pop in (0, 1):
            assert_obs_equal(gpu.obs(t, pop), ref.obs(t, pop), f"t={t} pop={pop}")


def test_adaptive_schedule(pa, oracle_lib):
    gpu, ref = make_pair(pa, oracle_lib, 6, 4000, None, n_temps=300, beta_max=3.0, eps_target=0.2, n_sweeps=3,
                         disorder_seed=5, run_seed=6)
    gpu.run()
    ref.run()
    assert gpu.t == ref.t
    for t in range(gpu.t + 1):
        assert gpu.beta(t) == ref.beta(t), t          # bitwise identical schedule
        assert_obs_equal(gpu.obs(t), ref.obs(t), f"adaptive t={t}")
    assert_state_equal(gpu, ref, 1, "adaptive end")


def test_sweep_schedule_and_zero_steps(pa, oracle_lib):
    betas = np.array([0.0, 0.3, 0.3, 0.9, 1.4, 1.4])
    sweeps = np.array([0, 0, 5, 1, 22, 3], dtype=np.int32)
    gpu, ref = make_pair(pa, oracle_lib, 4, 900, betas, sweeps_per_step=sweeps, disorder_seed=3, run_seed=4)
    gpu.run()
    ref.run()
    assert_state_equal(gpu, ref, 1, "sweep schedule")
    for t in range(6):
        assert_obs_equal(gpu.obs(t), ref.obs(t), f"t={t}")


def test_observables_read_while_the_next_step_runs(pa, oracle_lib):
    """pa_observables(t) waits for step t only: reading step t after step t + 1 (and
    t + 2) has been issued gives the oracle's step-t observables, for the adaptive
    schedule (whose pa_step reads the histogram itself) and an explicit one."""
    for betas in (None, linear(9, 2.0)):
        kw = dict(n_sweeps=2, disorder_seed=6, run_seed=9)
        if betas is None:
            gpu = pa.Run(8, 3000, 6, 9, None, n_temps=40, beta_max=2.0, eps_target=0.3, n_sweeps=2)
            ref = oracle_lib.Run(oracle_lib.RunConfig(L=8, R=3000, disorder_seed=6, run_seed=9, betas=None,
                                                      n_temps=40, beta_max=2.0, eps_target=0.3, n_sweeps=2))
        else:
            gpu, ref = make_pair(pa, oracle_lib, 8, 3000, betas, **kw)
        want = [ref.obs(0)]
        while ref.step() == 0:
            want.append(ref.obs(ref.t))
        got, t = [], 0
        while gpu.step() == 0:
            if gpu.t >= 2:
                got.append(gpu.obs(gpu.t - 2))   # two steps behind
            t = gpu.t
        for u in range(max(0, t - 1), t + 1):
            got.append(gpu.obs(u))
        assert t == ref.t and len(got) == len(want)
        for u, (g, r) in enumerate(zip(got, want)):
            assert_obs_equal(g, r, f"t={u}")
        assert_obs_equal(gpu.obs(1), want[1], "t=1 read last")   # an old step, whose own event was reused
        gpu.close()


def test_capacity_overflow_is_reported(pa, oracle_lib):
    betas = linear(6, 3.0)
    for run_seed in range(20):
        ref = oracle_lib.Run(oracle_lib.RunConfig(L=4, R=500, disorder_seed=1, run_seed=run_seed, betas=betas,
                                                  n_sweeps=1, R_cap=500))
        try:
            ref.run()
        except RuntimeError:
            break
    else:
        pytest.skip("no overflowing seed found")
    gpu = pa.Run(4, 500, 1, run_seed, betas, n_sweeps=1, R_cap=500)
    with pytest.raises(pa.PAError) as e:
        gpu.run()
    assert e.value.status == pa.PA_ERR_CAPACITY
    # the same error through the observables of each step (which wait for that step only)
    gpu = pa.Run(4, 500, 1, run_seed, betas, n_sweeps=1, R_cap=500)
    with pytest.raises(pa.PAError) as e:
        while gpu.step() == 0:
            gpu.obs(gpu.t)
    assert e.value.status == pa.PA_ERR_CAPACITY


def test_invalid_configurations_rejected(pa):
    with pytest.raises(pa.PAError):
        pa.Run(5, 10, 1, 1, linear(3, 1.0))            # odd L
    with pytest.raises(pa.PAError):
        pa.Run(66, 10, 1, 1, linear(3, 1.0))           # beyond the largest supported L (64)
    with pytest.raises(pa.PAError):
        pa.Run(4, 10, 1 << 56, 1, linear(3, 1.0))      # seed too large
    with pytest.raises(pa.PAError):
        pa.Run(4, 10, 1, 1, np.array([0.1, 0.2]))      # schedule must start at beta = 0
    with pytest.raises(pa.PAError):
        pa.Run(4, 10, 1, 1, np.array([0.0, 0.5, 0.2]))  # descending


def test_full_size_sampled_step(pa, oracle_lib):
    """L=10, R=1e6 (the large-population workload), two steps on the GPU in the
    launch configuration the benchmark times; sampled replicas are recomputed by
    the oracle one by one from their parents."""
    from paper_1711_02146_gb300.workloads import C3
    gpu = pa.Run.from_workload(C3)
    L, N = C3.L, C3.N
    J = gpu.couplings()
    assert np.array_equal(J, oracle_lib.couplings(L, C3.disorder_seed))
    rng = np.random.default_rng(0)
    for _ in range(2):
        s_old, lab_old, E_old = gpu.population()
        h_old = gpu.energy_hist(gpu.t)
        assert np.array_equal(np.bincount((E_old + 3 * N) // 2, minlength=3 * N + 1), h_old)
        for j in rng.integers(0, len(E_old), 16):
            assert oracle_lib.energy(L, J, s_old[j]) == E_old[j]
        gpu.step()
        t = gpu.t
        o = gpu.obs(t)
        # resampling: oracle tables from the GPU's integer histogram
        kmin, S, fl, thr, eps = oracle_lib.reweight(h_old, C3.R, o["dbeta"])
        assert o["kmin_prev"] == kmin and o["S_prime"] == S
        assert o["eps_expected"] == pytest.approx(eps, rel=REL)  # summed in another order on the device
        counts = gpu.copy_counts()
        assert counts.size == len(E_old)
        for i in rng.integers(0, len(E_old), 4000):
            k = (E_old[i] + 3 * N) // 2
            assert counts[i] == oracle_lib.copy_count(C3.run_seed, 0, t, int(i), int(fl[k]), int(thr[k]))
        parents = gpu.parents()
        assert parents.size == counts.sum() == o["R_tilde"]
        assert np.array_equal(parents, np.repeat(np.arange(len(E_old), dtype=np.int32), counts))
        s_new, lab_new, E_new = gpu.population()
        assert np.array_equal(lab_new, lab_old[parents])
        met = oracle_lib.metropolis_thresholds(gpu.beta(t))
        for j in rng.integers(0, len(E_new), 24):
            ref, dE = oracle_lib.sweep_replica(L, J, s_old[parents[j]], C3.run_seed, 0, int(j), t, C3.n_sweeps, met)
            assert np.array_equal(s_new[j], ref), f"slot {j}"
            assert E_new[j] == E_old[parents[j]] + dE
        assert np.array_equal(np.bincount((E_new + 3 * N) // 2, minlength=3 * N + 1), gpu.energy_hist(t))


@pytest.mark.parametrize("L,R,dbeta", [(4, 4_000_000, 0.4), (4, 4_000_000, 3.0), (2, 3_000_000, 0.0)])
def test_resampling_beyond_resident_tiles(pa, oracle_lib, L, R, dbeta):
    """More resampling tiles (R / 1024 > 2900) than the GPU holds at once, so the
    single-pass scan's later tiles start only after earlier ones have finished.
    First step out of beta = 0: sampled copy numbers (every tile's first and last
    slot among them) against the oracle's rule on the GPU's integer histogram, the
    whole parent map, the labels and R~; dbeta = 3 culls most replicas, dbeta = 0
    with R_{t-1} = R gives tau = 1 and so one copy of every replica."""
    gpu = pa.Run(L, R, 3, 11 + L, np.array([0.0, dbeta, dbeta + 0.5]), n_sweeps=1)
    N = L ** 3
    _, lab_old, E_old = gpu.population()
    h_old = gpu.energy_hist(0)
    assert gpu.step() == 0
    t, o = gpu.t, gpu.obs(gpu.t)
    assert t == 1
    kmin, S, fl, thr, eps = oracle_lib.reweight(h_old, R, o["dbeta"])
    assert o["kmin_prev"] == kmin and o["S_prime"] == S
    counts = gpu.copy_counts()
    assert counts.size == len(E_old) == R
    k = (E_old.astype(np.int64) + 3 * N) // 2
    rng = np.random.default_rng(5)
    for i in np.concatenate([rng.integers(0, R, 3000), np.arange(0, R, 1024), np.arange(1023, R, 1024), [R - 1]]):
        assert counts[i] == oracle_lib.copy_count(11 + L, 0, t, int(i), int(fl[k[i]]), int(thr[k[i]])), int(i)
    if dbeta == 0.0:
        assert np.all(counts == 1)
    parents = gpu.parents()
    assert parents.size == counts.sum() == o["R_tilde"]
    assert np.array_equal(parents, np.repeat(np.arange(R, dtype=np.int32), counts))
    _, lab_new, _ = gpu.population()
    assert np.array_equal(lab_new, lab_old[parents])
    assert o["culled"] == int((counts == 0).sum())


def test_c2_full_size_two_populations(pa, oracle_lib):
    """L = 8, R = 1e5, two populations (the overlap workload) at full size: the whole
    q histogram and I(0.2) recomputed from both GPU populations, and sampled replicas
    of population 1 swept again by the oracle (population index in the random key)."""
    from paper_1711_02146_gb300.workloads import C2
    gpu = pa.Run.from_workload(C2)
    L, N = C2.L, C2.N
    J = gpu.couplings()
    rng = np.random.default_rng(1)
    for _ in range(2):
        s_old, _, E_old = gpu.population(1)
        gpu.step()
        t = gpu.t
        A, B = gpu.population(0)[0], gpu.population(1)[0]
        pairs = min(A.shape[0], B.shape[0])
        Q = (A[:pairs].astype(np.int32) * B[:pairs].astype(np.int32)).sum(axis=1).astype(np.int64)
        bins = ((Q + N) * (C2.q_bins - 1) + N) // (2 * N)
        assert np.array_equal(np.bincount(bins, minlength=C2.q_bins), gpu.q_hist(t))
        o = gpu.obs(t, 0)
        assert o["q_pairs"] == pairs and o["q_abs_le_02"] == int((5 * np.abs(Q) <= N).sum())
        parents = gpu.parents(1)
        s_new, _, E_new = gpu.population(1)
        met = oracle_lib.metropolis_thresholds(gpu.beta(t))
        for j in rng.integers(0, len(E_new), 16):
            ref, dE = oracle_lib.sweep_replica(L, J, s_old[parents[j]], C2.run_seed, 1, int(j), t, C2.n_sweeps, met)
            assert np.array_equal(s_new[j], ref), f"pop 1 slot {j}"
            assert E_new[j] == E_old[parents[j]] + dE


def test_two_launch_sweep_for_a_partial_last_wave(pa, oracle_lib):
    """L = 10 with a population of 1.6e5: 157 tiles of 1024 replicas for 152 SMs, so the
    sweep runs the first 152 tiles with the 1024-replica shape and the rest with
    512-replica tiles in a second launch (when the device has 152 SMs; fewer SMs give
    other splits).  Every slot, energy, label and family statistic is the oracle's."""
    betas = linear(3, 0.8)
    gpu, ref = make_pair(pa, oracle_lib, 10, 160_000, betas, n_sweeps=1, disorder_seed=5, run_seed=8)
    if pa.sweep_selected(10) == 0 and _n_sm() == 152:
        assert gpu.sweep_plan() == {"shape": 0, "tail_shape": 1, "tail_from": 152 * 1024}
    for t in range(1, 3):
        assert gpu.step() == 0
        ref.step()
        assert np.array_equal(gpu.copy_counts(), ref.last_counts()), f"copy numbers at t={t}"
        assert np.array_equal(gpu.energy_hist(t), ref.energy_hist(t)), f"energy histogram at t={t}"
        assert_obs_equal(gpu.obs(t), ref.obs(t), f"t={t}")
    assert_state_equal(gpu, ref, 1, "two-launch sweep")


def _n_sm():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_sweep_plan_rule(pa):
    """The second launch is planned exactly when the run's R replicas fill at least
    one wave of tiles and leave a last wave at most 60 % full; it takes the next
    smaller tile and starts where the full waves end.  Gaussian runs, pinned shapes
    and runs among many have none."""
    n_sm = _n_sm()
    shapes = pa.sweep_shapes(10)
    pa.sweep_select(10, -1)
    for R in (1000, 100_000, 152 * 1024, 160_000, 250_000, 300_000, 1_000_000):
        run = pa.Run(10, R, 1, 2, linear(2, 0.5), n_sweeps=1)
        plan = run.sweep_plan()
        run.close()
        sh = shapes[plan["shape"]]
        tj = 32 * sh["words"]
        slots = n_sm * sh["ctas_per_sm"]
        tiles = -(-R // tj)
        full, rest = divmod(tiles, slots)
        smaller = [i for i, s in enumerate(shapes) if s["words"] < sh["words"]]
        if full >= 1 and rest > 0 and 10 * rest <= 6 * slots and smaller:
            best = max(smaller, key=lambda i: shapes[i]["words"])
            assert plan == {"shape": plan["shape"], "tail_shape": best, "tail_from": full * slots * tj}, R
            assert plan["tail_from"] % (32 * shapes[best]["words"]) == 0
        else:
            assert plan["tail_shape"] == -1 and plan["tail_from"] == 0, R
    pa.sweep_select(10, 0)   # pinned: one launch
    try:
        run = pa.Run(10, 160_000, 1, 2, linear(2, 0.5), n_sweeps=1)
        assert run.sweep_plan()["tail_shape"] == -1
        run.close()
    finally:
        pa.sweep_select(10, -1)
    g = pa.Run(10, 160_000, 1, 2, linear(2, 0.5), n_sweeps=1, model=pa.PA_MODEL_GAUSS)
    assert g.sweep_plan()["tail_shape"] == -1
    g.close()
