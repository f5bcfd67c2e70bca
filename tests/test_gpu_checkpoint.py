"""Checkpoint and restore (pa_checkpoint / pa_restore): a run restored at step t
and continued is bit-identical to the uninterrupted run; a checkpoint of another
configuration or a damaged buffer is refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02146_gb300 import build, pa as pa_mod
    build.build()
    return pa_mod


EXPLICIT = dict(L=6, R=700, disorder_seed=4, run_seed=9, betas=np.linspace(0.0, 2.5, 8), n_sweeps=2, n_pop=2)
ADAPTIVE = dict(L=4, R=500, disorder_seed=2, run_seed=5, betas=None, n_temps=200, beta_max=3.0, eps_target=0.3,
                n_sweeps=2)


def make(pa, kw, **extra):
    kw = dict(kw)
    return pa.Run(kw.pop("L"), kw.pop("R"), kw.pop("disorder_seed"), kw.pop("run_seed"), kw.pop("betas"), **kw,
                  **extra)


def trace(run, upto=None):
    """Everything observable after the run's last step."""
    t = run.t
    out = {"t": t, "obs": [[run.obs(u, p) for p in range(run.n_pop)] for u in range(t + 1)],
           "hist": [[run.energy_hist(u, p) for p in range(run.n_pop)] for u in range(t + 1)],
           "pop": [run.population(p) for p in range(run.n_pop)],
           "fam": [run.family_hist(p) for p in range(run.n_pop)]}
    if run.n_pop == 2:
        out["q"] = [run.q_hist(u) for u in range(t + 1)]
    if t > 0:
        out["counts"] = [run.copy_counts(p) for p in range(run.n_pop)]
        out["parents"] = [run.parents(p) for p in range(run.n_pop)]
    return out


def assert_same(a, b):
    assert a["t"] == b["t"]
    assert a["obs"] == b["obs"]
    for x, y in zip(a["hist"], b["hist"]):
        assert all(np.array_equal(u, v) for u, v in zip(x, y))
    for x, y in zip(a["pop"], b["pop"]):
        assert all(np.array_equal(u, v) for u, v in zip(x, y))
    for x, y in zip(a["fam"], b["fam"]):
        assert all(np.array_equal(u, v) for u, v in zip(x, y))
    for k in ("q", "counts", "parents"):
        if k in a:
            assert all(np.array_equal(u, v) for u, v in zip(a[k], b[k]))


@pytest.mark.parametrize("kw,at", [(EXPLICIT, 3), (EXPLICIT, 0), (ADAPTIVE, 2)])
def test_restored_run_continues_bit_identically(pa, kw, at):
    ref = make(pa, kw)
    ref.run()
    full = trace(ref)
    ref.close()

    first = make(pa, kw)
    for _ in range(at):
        assert first.step() == 0
    blob = first.checkpoint()
    before = trace(first)
    first.close()

    resumed = make(pa, kw, checkpoint=blob)
    assert resumed.t == at
    assert_same(trace(resumed), before)         # the state itself came back
    resumed.run()
    assert_same(trace(resumed), full)           # and the continuation is the uninterrupted run
    resumed.close()


def test_checkpoint_of_a_finished_run(pa):
    run = make(pa, EXPLICIT)
    run.run()
    blob = run.checkpoint()
    again = make(pa, EXPLICIT, checkpoint=blob)
    assert again.step() == pa.PA_DONE
    assert_same(trace(again), trace(run))


def test_refuses_other_configurations_and_damaged_buffers(pa):
    run = make(pa, EXPLICIT)
    run.step()
    blob = run.checkpoint()
    for change in (dict(run_seed=10), dict(disorder_seed=5), dict(R=701), dict(n_sweeps=3),
                   dict(betas=np.linspace(0.0, 2.6, 8))):
        with pytest.raises(pa.PAError) as e:
            make(pa, {**EXPLICIT, **change}, checkpoint=blob)
        assert e.value.status == pa.PA_ERR_INVALID
    for bad in (blob[:-1], blob + b"\0", b"XXXXXXXX" + blob[8:]):
        with pytest.raises(pa.PAError) as e:
            make(pa, EXPLICIT, checkpoint=bad)
        assert e.value.status == pa.PA_ERR_INVALID
    import ctypes
    n = ctypes.c_size_t()
    small = ctypes.create_string_buffer(16)
    assert pa.lib().pa_checkpoint(run._h, small, 16, ctypes.byref(n)) == pa.PA_ERR_CAPACITY
    assert n.value == len(blob)


GAUSS = dict(L=6, R=800, disorder_seed=3, run_seed=8, betas=np.linspace(0.0, 2.5, 7), n_sweeps=2, n_pop=2)
GAUSS_ADAPTIVE = dict(L=4, R=600, disorder_seed=5, run_seed=6, betas=None, n_temps=300, beta_max=2.0,
                      eps_target=0.3, n_sweeps=2)


def gtrace(run):
    """Everything observable of a Gaussian-coupling run after its last step."""
    t = run.t
    out = {"t": t, "obs": [[run.gobs(u, p) for p in range(run.n_pop)] for u in range(t + 1)],
           "pop": [run.population(p) for p in range(run.n_pop)],
           "fam": [run.family_hist(p) for p in range(run.n_pop)]}
    if run.n_pop == 2:
        out["q"] = [run.q_hist(u) for u in range(t + 1)]
        out["ql"] = [run.ql_hist(u) for u in range(t + 1)]
    if t > 0:
        out["counts"] = [run.copy_counts(p) for p in range(run.n_pop)]
        out["parents"] = [run.parents(p) for p in range(run.n_pop)]
    return out


def assert_gsame(a, b):
    assert a["t"] == b["t"]
    assert a["obs"] == b["obs"]
    for x, y in zip(a["pop"], b["pop"]):
        assert all(np.array_equal(u, v) for u, v in zip(x, y))
    for x, y in zip(a["fam"], b["fam"]):
        assert all(np.array_equal(u, v) for u, v in zip(x, y))
    for k in ("q", "ql", "counts", "parents"):
        if k in a:
            assert all(np.array_equal(u, v) for u, v in zip(a[k], b[k]))


@pytest.mark.parametrize("kw,at", [(GAUSS, 3), (GAUSS, 0), (GAUSS_ADAPTIVE, 2)])
def test_gaussian_run_restored_continues_bit_identically(pa, kw, at):
    ref = make(pa, kw, model=pa.PA_MODEL_GAUSS)
    ref.run()
    full = gtrace(ref)
    ref.close()

    first = make(pa, kw, model=pa.PA_MODEL_GAUSS)
    for _ in range(at):
        assert first.step() == 0
    blob = first.checkpoint()
    before = gtrace(first)
    first.close()

    resumed = make(pa, kw, model=pa.PA_MODEL_GAUSS, checkpoint=blob)
    assert resumed.t == at
    assert_gsame(gtrace(resumed), before)
    resumed.run()
    assert_gsame(gtrace(resumed), full)
    resumed.close()


def test_checkpoint_of_one_model_is_refused_by_the_other(pa):
    g = make(pa, GAUSS, model=pa.PA_MODEL_GAUSS)
    g.step()
    blob = g.checkpoint()
    with pytest.raises(pa.PAError) as e:
        make(pa, GAUSS, checkpoint=blob)            # same sizes, +-1 couplings
    assert e.value.status == pa.PA_ERR_INVALID
    p = make(pa, GAUSS)
    p.step()
    with pytest.raises(pa.PAError) as e:
        make(pa, GAUSS, model=pa.PA_MODEL_GAUSS, checkpoint=p.checkpoint())
    assert e.value.status == pa.PA_ERR_INVALID
