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
