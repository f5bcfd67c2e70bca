"""The allocation-free resampling entry point against pa_step's own resampling.

pa_resample_counts_noalloc serves callers that cannot allocate device memory
(code under a framework allocator that owns the device memory, latency-critical
loops where cudaMalloc would synchronise, exactly budgeted deployments): its
scratch is a fixed array inside the library.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02146_gb300 import build, pa
    build.build()
    return torch, pa


def test_noalloc_resampling_matches_pa_step(env, oracle_lib):
    torch, pa = env
    L, R, disorder_seed, run_seed = 6, 5000, 3, 4
    N = L ** 3
    betas = np.array([t * 1.5 / 3 for t in range(4)])
    run = pa.Run(L, R, disorder_seed, run_seed, betas, n_sweeps=2)
    dev = torch.device("cuda")
    for _ in range(2):  # two calls in a row, on two successive resamplings
        _, _, E_old = run.population()
        hist = run.energy_hist(run.t)
        t = run.t + 1
        assert run.step() == 0
        counts_ref = run.copy_counts()
        parents_ref = run.parents()
        # the reweighting tables pa_step used (bit-identical to the GPU's, see the parity tests)
        _, _, fl, thr, _ = oracle_lib.reweight(hist, R, run.beta(t) - run.beta(t - 1))
        levels = torch.from_numpy(((E_old + 3 * N) // 2).astype(np.int32)).to(dev)
        fl_d = torch.from_numpy(fl.astype(np.int32)).to(dev)
        thr_d = torch.from_numpy(thr.astype(np.uint32).view(np.int32)).to(dev)
        n_old = len(E_old)
        cap = len(parents_ref) + 64
        counts = torch.full((n_old,), -1, dtype=torch.int32, device=dev)
        parents = torch.full((cap,), -1, dtype=torch.int32, device=dev)
        n_new = torch.zeros(1, dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        rc = pa.resample_counts_noalloc(levels.data_ptr(), n_old, fl_d.data_ptr(), thr_d.data_ptr(), 3 * N + 1,
                                        run_seed, 0, t, counts.data_ptr(), parents.data_ptr(), cap, n_new.data_ptr(),
                                        torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert rc == pa.PA_OK
        assert np.array_equal(counts.cpu().numpy(), counts_ref)
        assert int(n_new.item()) == len(parents_ref)
        p = parents.cpu().numpy()
        assert np.array_equal(p[:len(parents_ref)], parents_ref)
        assert np.all(p[len(parents_ref):] == -1)  # nothing written past the new population


def test_noalloc_rejects_inputs_beyond_its_scratch(env):
    torch, pa = env
    n_new = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = pa.resample_counts_noalloc(0, pa.NOALLOC_MAX_SLOTS + 1, 0, 0, 10, 1, 0, 1, 0, 0, 0, n_new.data_ptr())
    assert rc == pa.PA_ERR_INVALID


def _call(torch, pa, levels, fl, thr, n_levels, run_seed, t, cap, guard=1024):
    """One call on fresh device copies; parents sit between two guard zones of -1."""
    dev = torch.device("cuda")
    levels_d = torch.from_numpy(np.ascontiguousarray(levels, np.int32)).to(dev)
    fl_d = torch.from_numpy(np.ascontiguousarray(fl, np.int32)).to(dev)
    thr_d = torch.from_numpy(np.ascontiguousarray(thr, np.uint32).view(np.int32)).to(dev)
    n_old = levels.size
    counts = torch.full((n_old,), -7, dtype=torch.int32, device=dev)
    buf = torch.full((cap + 2 * guard,), -1, dtype=torch.int32, device=dev)
    n_new = torch.zeros(1, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    rc = pa.resample_counts_noalloc(levels_d.data_ptr(), n_old, fl_d.data_ptr(), thr_d.data_ptr(), n_levels, run_seed,
                                    0, t, counts.data_ptr(), buf.data_ptr() + 4 * guard, cap, n_new.data_ptr(),
                                    torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert rc == pa.PA_OK
    b = buf.cpu().numpy()
    assert np.all(b[:guard] == -1) and np.all(b[guard + cap:] == -1), "write outside parents[0, cap)"
    return counts.cpu().numpy(), int(n_new.item()), b[guard:guard + cap]


def test_noalloc_many_blocks_against_the_oracle(env, oracle_lib):
    """3e6 old slots (2930 blocks, so the one-block scan carries over three rounds of
    1024 block totals), synthetic levels and tables: every copy number against the
    oracle's nearest-integer rule, the total, and the whole parent map (the
    concatenation of n_i copies of each old slot in slot order), twice in a row."""
    torch, pa = env
    rng = np.random.default_rng(11)
    n_old, n_levels, run_seed = 3_000_000, 3001, 77
    levels = rng.integers(0, n_levels, n_old).astype(np.int32)
    fl = rng.integers(0, 4, n_levels).astype(np.int32)
    thr = rng.integers(0, 2 ** 32, n_levels, dtype=np.uint64).astype(np.uint32)
    for t in (5, 6):
        want = oracle_lib.copy_counts(run_seed, 0, t, levels, fl, thr)
        total = int(want.astype(np.int64).sum())
        counts, n_new, parents = _call(torch, pa, levels, fl, thr, n_levels, run_seed, t, total + 100)
        assert np.array_equal(counts, want)
        assert n_new == total
        assert np.array_equal(parents[:total], np.repeat(np.arange(n_old, dtype=np.int32), want))
        assert np.all(parents[total:] == -1)


def test_noalloc_totals_beyond_32_bits(env, oracle_lib):
    """2.5e6 old slots with 1000 or 1001 copies each: the new population size
    (about 2.5e9) exceeds 2^31 - 1 and is reported exactly; only parents[0, cap)
    are written."""
    torch, pa = env
    n_old, run_seed, t, cap = 2_500_000, 5, 3, 5000
    levels = (np.arange(n_old) % 7).astype(np.int32)
    fl = np.full(7, 1000, np.int32)
    thr = np.array([0, 2 ** 31, 2 ** 32 - 1, 1, 3 * 2 ** 30, 2 ** 30, 12345], np.uint32)
    want = oracle_lib.copy_counts(run_seed, 0, t, levels, fl, thr)
    counts, n_new, parents = _call(torch, pa, levels, fl, thr, 7, run_seed, t, cap)
    assert np.array_equal(counts, want)
    assert n_new == int(want.astype(np.int64).sum()) > 2 ** 31
    assert np.array_equal(parents, np.repeat(np.arange(8, dtype=np.int32), want[:8])[:cap])


@pytest.mark.parametrize("case", ["negative floor", "level above the tables", "negative level"])
def test_noalloc_reports_invalid_device_data(env, case):
    """Bad table or level entries are reported on the device (*n_new = -1) and no
    parent is written; the next valid call is unaffected."""
    torch, pa = env
    rng = np.random.default_rng(3)
    n_old, n_levels = 5000, 50
    levels = rng.integers(0, n_levels, n_old).astype(np.int32)
    fl = np.ones(n_levels, np.int32)
    thr = np.zeros(n_levels, np.uint32)
    if case == "negative floor":
        fl[levels[4321]] = -5
    elif case == "level above the tables":
        levels[4321] = n_levels
    else:
        levels[17] = -1
    _, n_new, parents = _call(torch, pa, levels, fl, thr, n_levels, 9, 1, 2 * n_old)
    assert n_new == -1
    assert np.all(parents == -1)
    ok_levels = np.clip(levels, 0, n_levels - 1)
    counts, n_new, parents = _call(torch, pa, ok_levels, np.ones(n_levels, np.int32), thr, n_levels, 9, 1, 2 * n_old)
    assert n_new == n_old and np.all(counts == 1)
    assert np.array_equal(parents[:n_old], np.arange(n_old, dtype=np.int32))
