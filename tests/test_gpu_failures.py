"""Failure detection on the GPU without a fault: the single-pass resampling (§II)
waits for its predecessor tiles' entries with a bounded number of polls.  A test
hook withholds one tile's entries (a flag that nothing sets) and lowers the poll
limit, so that the waits after it run out: the kernel ends normally with the
timeout flag set, the run reports PA_ERR_TIMEOUT, and the GPU and later runs are
unaffected (bit-exact with the oracle afterwards)."""
import numpy as np
import pytest

from test_gpu_parity import assert_obs_equal, assert_state_equal, linear, make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02146_gb300 import build, pa as pa_mod
    build.build()
    return pa_mod


def test_lookback_wait_runs_out_and_is_reported(pa, oracle_lib):
    betas = linear(4, 1.5)
    run = pa.Run(6, 5000, 3, 4, betas, n_sweeps=2)   # 5000 old slots: five tiles of 1024
    assert pa.lib().pa_debug_lookback(run._h, 64, 1) == pa.PA_OK
    try:
        run.step()
        run.sync()
    except pa.PAError as e:
        assert e.status == pa.PA_ERR_TIMEOUT
    else:
        pytest.fail("the withheld tile's successors did not report a timeout")
    for call in (run.sync, run.step, lambda: run.obs(1)):
        with pytest.raises(pa.PAError) as e:
            call()
        assert e.value.status == pa.PA_ERR_TIMEOUT
    # the same configuration on the same GPU afterwards: the oracle's results bit for bit
    gpu, ref = make_pair(pa, oracle_lib, 6, 5000, betas, n_sweeps=2, disorder_seed=3, run_seed=4)
    for t in range(1, len(betas)):
        assert gpu.step() == 0
        ref.step()
        assert np.array_equal(gpu.copy_counts(), ref.last_counts()), f"copy numbers at t={t}"
        assert_obs_equal(gpu.obs(t), ref.obs(t), f"t={t}")
    assert_state_equal(gpu, ref, 1, "after the timed-out run")


def test_lookback_hook_restores_the_default(pa, oracle_lib):
    betas = linear(3, 1.0)
    gpu, ref = make_pair(pa, oracle_lib, 4, 3000, betas, n_sweeps=2, disorder_seed=2, run_seed=5)
    lib = pa.lib()
    assert lib.pa_debug_lookback(gpu._h, -1, -1) == pa.PA_ERR_INVALID
    assert lib.pa_debug_lookback(gpu._h, 5, -2) == pa.PA_ERR_INVALID
    assert lib.pa_debug_lookback(gpu._h, 64, 0) == pa.PA_OK
    assert lib.pa_debug_lookback(gpu._h, 0, -1) == pa.PA_OK   # back to the default limit, nothing withheld
    gpu.run()
    ref.run()
    assert_state_equal(gpu, ref, 1, "default look-back")
    assert_obs_equal(gpu.obs(2), ref.obs(2), "t=2")


def test_bisection_barrier_wait_runs_out_and_is_reported(pa):
    """The one-launch bisection of a Gaussian-coupling run (§IV.B): one block is kept
    from the first grid barrier (a flag that nothing sets) and the poll limit lowered,
    so the other blocks' waits run out; the launch ends normally with its error set,
    the run reports PA_ERR_TIMEOUT from then on, and a run afterwards on the same GPU
    is the same to the bit as one made before."""
    cfg = dict(n_temps=80, beta_max=2.0, eps_target=0.3, n_sweeps=1, model=pa.PA_MODEL_GAUSS)
    before = pa.Run(6, 3000, 5, 76, None, **cfg)
    before.run()
    bad = pa.Run(6, 3000, 5, 76, None, **cfg)
    assert pa.lib().pa_debug_bisect(bad._h, 1, 0) == pa.PA_OK
    for call in (bad.step, bad.sync, bad.step):
        with pytest.raises(pa.PAError) as e:
            call()
        assert e.value.status == pa.PA_ERR_TIMEOUT
    after = pa.Run(6, 3000, 5, 76, None, **cfg)
    after.run()
    assert before.t == after.t >= 3
    for t in range(before.t + 1):
        assert before.gobs(t) == after.gobs(t) or all(
            a == b or (a != a and b != b) for a, b in zip(before.gobs(t).values(), after.gobs(t).values())), t
    for x, y in zip(before.population(), after.population()):
        assert np.array_equal(x, y)
    for r in (before, bad, after):
        r.close()
