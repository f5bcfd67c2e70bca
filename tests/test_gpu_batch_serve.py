"""Batched and served runs (pa_batch, pa_server): every run gives exactly the
result it gives alone, whatever else shares the GPU; admission respects the
memory budget; a failing request does not disturb the others."""
import time

import numpy as np
import pytest

from paper_1711_02146_gb300.workloads import Workload, linear_betas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02146_gb300 import build, pa as pa_mod
    build.build()
    return pa_mod


def mixed_workloads(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        L = [4, 6, 8, 10][i % 4]
        R = int(rng.integers(300, 3000))
        T = int(rng.integers(4, 12))
        out.append(Workload(f"mix{i}", L=L, R=R, disorder_seed=500 + i, run_seed=900 + i,
                            betas=linear_betas(T, 2.5), n_sweeps=int(rng.integers(1, 4)), n_pop=1 + (i % 3 == 0)))
    return out


def standalone(pa, w):
    r = pa.Run.from_workload(w)
    r.run()
    return r


def assert_same_run(a, b, w, every_step=False):
    t = a.t
    assert b.t == t
    for u in (range(t + 1) if every_step else (t,)):
        for pop in range(w.n_pop):
            assert a.obs(u, pop) == b.obs(u, pop), f"{w.name} t={u} pop {pop}"
            assert np.array_equal(a.energy_hist(u, pop), b.energy_hist(u, pop)), f"{w.name} t={u}"
        if w.n_pop == 2:
            assert np.array_equal(a.q_hist(u), b.q_hist(u)), f"{w.name} t={u}"
    for pop in range(w.n_pop):
        sa, la, ea = a.population(pop)
        sb, lb, eb = b.population(pop)
        assert np.array_equal(sa, sb) and np.array_equal(la, lb) and np.array_equal(ea, eb)
        assert np.array_equal(a.copy_counts(pop), b.copy_counts(pop))


@pytest.mark.parametrize("mode", ["fused", "streams"])
def test_batch_matches_standalone_runs(pa, mode):
    ws = mixed_workloads(9)
    batch = pa.Batch(ws, mode=mode)
    batch.run()
    for i, w in enumerate(ws):
        assert_same_run(batch.run_view(i), standalone(pa, w), w, every_step=True)
    n = batch.launches()
    if mode == "fused":   # 11 rounds (the longest schedule), one graph launch each
        rounds = max(len(w.betas) for w in ws) - 1
        assert n["graphs"] == rounds and n["kernels"] == rounds * (3 + 4 + 1)
    else:
        assert n["graphs"] == 0 and n["kernels"] > 0
    batch.close()


def test_fused_batch_every_size_and_shape(pa):
    """The fused rounds with every lattice size of the shared-memory sweep,
    populations of many tiles and many resampling blocks, two-population runs, schedules of different lengths (runs
    that finish early rest), a run already stepped alone before the batch runs, and
    runs that do not qualify (Gaussian couplings, an adaptive schedule, L = 18) beside
    them: every run, every step, exactly as alone."""
    ws = [Workload("a4", L=4, R=5000, disorder_seed=11, run_seed=12, betas=linear_betas(9, 3.0), n_sweeps=2),
          Workload("a6", L=6, R=20000, disorder_seed=13, run_seed=14, betas=linear_betas(5, 1.5), n_sweeps=1),
          Workload("a8p", L=8, R=9000, disorder_seed=15, run_seed=16, betas=linear_betas(7, 2.0), n_sweeps=2,
                   n_pop=2),
          Workload("a10", L=10, R=30000, disorder_seed=17, run_seed=18, betas=linear_betas(4, 1.0), n_sweeps=1),
          Workload("a12", L=12, R=3000, disorder_seed=19, run_seed=20, betas=linear_betas(6, 2.5), n_sweeps=1),
          Workload("a14", L=14, R=1500, disorder_seed=21, run_seed=22, betas=linear_betas(3, 1.0), n_sweeps=1),
          Workload("a16", L=16, R=1100, disorder_seed=23, run_seed=24, betas=linear_betas(3, 0.6), n_sweeps=1,
                   n_pop=2),
          Workload("a10b", L=10, R=700, disorder_seed=25, run_seed=26, betas=linear_betas(8, 4.0), n_sweeps=3),
          Workload("ga", L=6, R=800, disorder_seed=27, run_seed=28, betas=linear_betas(5, 2.0), n_sweeps=2, model=1),
          Workload("ad", L=6, R=2000, disorder_seed=29, run_seed=30, betas=None, beta_max=2.0, eps_target=0.3,
                   n_temps=60, n_sweeps=2),
          Workload("g18", L=18, R=600, disorder_seed=31, run_seed=32, betas=linear_betas(3, 0.8), n_sweeps=1)]
    batch = pa.Batch(ws)
    batch.run_view(1).step()   # a6 starts the rounds at t = 1
    batch.run()
    for i, w in enumerate(ws):
        a, b = batch.run_view(i), standalone(pa, w)
        if w.model == 1:
            t = a.t
            assert b.t == t
            for x, y in zip(a.population(0), b.population(0)):
                assert np.array_equal(x, y)
            assert a.gobs(t) == b.gobs(t)
        else:
            assert_same_run(a, b, w, every_step=True)
    n = batch.launches()
    assert n["graphs"] == 8   # a4: 8 steps
    batch.close()


def drain(server, ids, limit_s=120.0):
    done = set()
    t0 = time.time()
    while len(done) < len(ids):
        done.update(server.poll())
        assert time.time() - t0 < limit_s, "server did not finish"
    return done


def test_server_results_identical_alone_and_in_the_mix(pa):
    ws = mixed_workloads(12, seed=1)
    budget = int(2.2 * max(pa.footprint(w) for w in ws))
    server = pa.Server(budget, max_active=6, steps_per_poll=2)
    ids = [server.submit(w) for w in ws]
    peak_active = 0
    done = set()
    t0 = time.time()
    while len(done) < len(ids):
        done.update(server.poll())
        q, a = server.load()
        peak_active = max(peak_active, a)
        assert a <= 6
        assert time.time() - t0 < 120.0
    assert peak_active >= 2           # requests did overlap on the device
    for rid, w in zip(ids, ws):
        ref = standalone(pa, w)
        for pop in range(w.n_pop):
            obs, last = server.result(rid, pop)
            assert last == ref.t
            assert obs == ref.obs(ref.t, pop)
    server.close()


def test_server_isolates_a_failing_request(pa, oracle_lib):
    betas = linear_betas(6, 3.0)
    for run_seed in range(30):  # a seed whose population outgrows a capacity equal to R
        ref = oracle_lib.Run(oracle_lib.RunConfig(L=4, R=500, disorder_seed=1, run_seed=run_seed, betas=betas,
                                                  n_sweeps=1, R_cap=500))
        try:
            ref.run()
        except RuntimeError:
            break
    else:
        pytest.skip("no overflowing seed found")
    bad = Workload("bad", L=4, R=500, disorder_seed=1, run_seed=run_seed, betas=betas, n_sweeps=1, R_cap=500)
    good = mixed_workloads(5, seed=2)
    server = pa.Server(int(1e10), max_active=8)
    ids = [server.submit(w) for w in good[:2]] + [server.submit(bad)] + [server.submit(w) for w in good[2:]]
    drain(server, ids)
    with pytest.raises(pa.PAError) as e:
        server.result(ids[2])
    assert e.value.status == pa.PA_ERR_CAPACITY
    for rid, w in zip(ids[:2] + ids[3:], good):
        ref = standalone(pa, w)
        obs, last = server.result(rid)
        assert last == ref.t and obs == ref.obs(ref.t)
    server.close()


@pytest.mark.parametrize("mode", ["fused", "streams"])
def test_batch_reports_a_failing_run_and_finishes_the_others(pa, oracle_lib, mode):
    """A run whose population outgrows a capacity equal to R, in a batch: pa_batch_run
    reports PA_ERR_CAPACITY (from the run's device flag), the run itself reports it,
    and every other run of the batch gives its standalone results, every step."""
    betas = linear_betas(6, 3.0)
    for run_seed in range(30):  # a seed whose population outgrows a capacity equal to R
        ref = oracle_lib.Run(oracle_lib.RunConfig(L=4, R=500, disorder_seed=1, run_seed=run_seed, betas=betas,
                                                  n_sweeps=1, R_cap=500))
        try:
            ref.run()
        except RuntimeError:
            break
    else:
        pytest.skip("no overflowing seed found")
    bad = Workload("bad", L=4, R=500, disorder_seed=1, run_seed=run_seed, betas=betas, n_sweeps=1, R_cap=500)
    good = mixed_workloads(5, seed=3)
    ws = good[:2] + [bad] + good[2:]
    batch = pa.Batch(ws, mode=mode)
    with pytest.raises(pa.PAError) as e:
        batch.run()
    assert e.value.status == pa.PA_ERR_CAPACITY
    with pytest.raises(pa.PAError) as e:
        batch.run_view(2).sync()
    assert e.value.status == pa.PA_ERR_CAPACITY
    for i, w in enumerate(ws):
        if w is not bad:
            assert_same_run(batch.run_view(i), standalone(pa, w), w, every_step=True)
    batch.close()


def test_server_rejects_requests_beyond_the_budget(pa):
    from paper_1711_02146_gb300.workloads import C1
    server = pa.Server(1000)
    with pytest.raises(pa.PAError) as e:
        server.submit(C1)
    assert e.value.status == pa.PA_ERR_NOMEM
    server.close()


def test_batch_mixes_models(pa):
    """Gaussian and +-1 runs in one batch give exactly their standalone results."""
    ws = [Workload("pm", L=6, R=900, disorder_seed=3, run_seed=4, betas=linear_betas(6, 2.0), n_sweeps=2),
          Workload("ga", L=8, R=700, disorder_seed=5, run_seed=6, betas=linear_betas(7, 2.5), n_sweeps=2, model=1),
          Workload("ga2", L=4, R=1500, disorder_seed=7, run_seed=8, betas=linear_betas(5, 1.5), n_sweeps=3,
                   n_pop=2, model=1)]
    batch = pa.Batch(ws)
    batch.run()
    for i, w in enumerate(ws):
        a, b = batch.run_view(i), standalone(pa, w)
        if w.model == 0:
            assert_same_run(a, b, w)
            continue
        t = a.t
        assert b.t == t
        for pop in range(w.n_pop):
            assert a.gobs(t, pop) == b.gobs(t, pop)
            for x, y in zip(a.population(pop), b.population(pop)):
                assert np.array_equal(x, y)
        if w.n_pop == 2:
            assert np.array_equal(a.ql_hist(t), b.ql_hist(t))
    batch.close()


def test_server_serves_both_models(pa):
    """Gaussian and +-1 requests in one server: each result equals its standalone
    run's, and each model's reader refuses the other's requests."""
    ws = [Workload("pm", L=6, R=900, disorder_seed=3, run_seed=4, betas=linear_betas(6, 2.0), n_sweeps=2),
          Workload("ga", L=8, R=700, disorder_seed=5, run_seed=6, betas=linear_betas(7, 2.5), n_sweeps=2, model=1),
          Workload("ga2", L=4, R=1500, disorder_seed=7, run_seed=8, betas=linear_betas(5, 1.5), n_sweeps=3,
                   n_pop=2, model=1),
          Workload("pm2", L=4, R=2000, disorder_seed=9, run_seed=10, betas=linear_betas(9, 3.0), n_sweeps=2,
                   n_pop=2)]
    budget = int(3 * max(pa.footprint(w) for w in ws))
    server = pa.Server(budget, max_active=4, steps_per_poll=2)
    ids = [server.submit(w) for w in ws]
    done, t0 = set(), time.time()
    while len(done) < len(ids):
        done.update(server.poll())
        assert time.time() - t0 < 120.0
    for rid, w in zip(ids, ws):
        ref = standalone(pa, w)
        for pop in range(w.n_pop):
            if w.model == 1:
                obs, last = server.gresult(rid, pop)
                assert last == ref.t and obs == ref.gobs(ref.t, pop)
                with pytest.raises(pa.PAError):
                    server.result(rid, pop)
            else:
                obs, last = server.result(rid, pop)
                assert last == ref.t and obs == ref.obs(ref.t, pop)
                with pytest.raises(pa.PAError):
                    server.gresult(rid, pop)
    server.close()
