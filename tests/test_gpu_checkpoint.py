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


def _sections(blob, run, t, n_temps, n_levels, gauss=False):
    """Byte offsets of population 0's sections in a checkpoint taken at step t (the
    layout pa_checkpoint writes: header, schedule, then per population the step
    records, level histograms or Gaussian records, spins, labels, levels or
    energies, copy numbers, parents, family-size histogram)."""
    header = int(np.frombuffer(blob[12:16], np.uint32)[0])
    Rt, Rp = len(run.population(0)[1]), len(run.copy_counts(0))
    off, out = header + 12 * n_temps, {}
    sizes = [("rec", 88 * (t + 1)), ("hist", (64 if gauss else 4 * n_levels) * (t + 1)), ("spins", run.N * Rt),
             ("labels", 4 * Rt), ("levels", (8 if gauss else 4) * Rt), ("counts", 4 * Rp), ("parents", 4 * Rt),
             ("mhist", 4 * (Rt + 1))]
    for name, size in sizes:
        out[name] = (off, size)
        off += size
    return out, Rt, Rp


def _put(blob, at, dtype, value):
    b = bytearray(blob)
    b[at:at + np.dtype(dtype).itemsize] = np.array([value], dtype=dtype).tobytes()
    return bytes(b)


def test_refuses_damaged_contents(pa):
    """A buffer of the right size whose contents were damaged is refused before any of
    it reaches the device: every value a kernel uses as an index or a size is checked
    on the host (records, histograms, spins, labels, levels, copy numbers, parents,
    family sizes)."""
    from paper_1711_02146_gb300.workloads import default_capacity
    t = 3
    run = make(pa, EXPLICIT)
    for _ in range(t):
        run.step()
    blob = run.checkpoint()
    n_levels = 3 * run.N + 1
    sec, Rt, Rp = _sections(blob, run, t, len(EXPLICIT["betas"]), n_levels)
    rec, hist, spins = sec["rec"][0], sec["hist"][0], sec["spins"][0]
    lab, lev, cnt, par, mh = (sec[k][0] for k in ("labels", "levels", "counts", "parents", "mhist"))
    levels0 = np.frombuffer(blob[lev:lev + 4 * Rt], np.int32)
    other = int(levels0[0] + 1 if levels0[0] + 1 < n_levels else levels0[0] - 1)
    damaged = {
        "R_tilde of the last record": _put(blob, rec + 88 * t, np.int32, default_capacity(EXPLICIT["R"]) + 5),
        "R_prev of a record": _put(blob, rec + 88 * 2 + 4, np.int32, 3),
        "lowest level of a record": _put(blob, rec + 88 * 1 + 8, np.int32, n_levels),
        "a histogram bin": _put(blob, hist + 4 * (t * n_levels + 7), np.uint32, 99),
        "a spin byte": _put(blob, spins + 1234, np.int8, 0),
        "a label above R": _put(blob, lab + 4 * (Rt - 1), np.int32, EXPLICIT["R"]),
        "a descending label": _put(blob, lab, np.int32, EXPLICIT["R"] - 1),
        "a level beyond the table": _put(blob, lev + 4 * 5, np.int32, n_levels),
        "a level not in the histogram": _put(blob, lev, np.int32, other),
        "a negative copy number": _put(blob, cnt + 4 * 9, np.int32, -1),
        "a parent beyond the old population": _put(blob, par + 4 * (Rt - 1), np.int32, Rp),
        "a family-size count": _put(blob, mh + 4 * 1, np.int32, -4),
    }
    for what, bad in damaged.items():
        assert len(bad) == len(blob) and bad != blob, what
        with pytest.raises(pa.PAError) as e:
            make(pa, EXPLICIT, checkpoint=bad)
        assert e.value.status == pa.PA_ERR_INVALID, what
    restored = make(pa, EXPLICIT, checkpoint=blob)
    assert_same(trace(restored), trace(run))
    gr = make(pa, GAUSS, model=pa.PA_MODEL_GAUSS)
    for _ in range(2):
        gr.step()
    gblob = gr.checkpoint()
    gsec, gRt, _ = _sections(gblob, gr, 2, len(GAUSS["betas"]), 0, gauss=True)
    for what, bad in {"an energy below the lowest": _put(gblob, gsec["levels"][0], np.int64, -(2 ** 40)),
                      "a label above R": _put(gblob, gsec["labels"][0] + 4 * (gRt - 1), np.int32, GAUSS["R"])}.items():
        with pytest.raises(pa.PAError) as e:
            make(pa, GAUSS, model=pa.PA_MODEL_GAUSS, checkpoint=bad)
        assert e.value.status == pa.PA_ERR_INVALID, what


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
