"""Every compiled launch shape of the sweep kernel gives the oracle's results bit
for bit (the random words depend on slot and site only), and the autotuner
selects one of them without changing any result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIZES = [(2, 301), (4, 700), (6, 555), (8, 1100), (10, 515), (12, 300), (14, 129), (16, 65)]


@pytest.fixture(scope="module")
def pa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02146_gb300 import build, pa as pa_mod
    build.build()
    yield pa_mod
    for L, _ in SIZES:
        pa_mod.sweep_select(L, -1)


def oracle_trace(oracle_lib, L, R, betas, S):
    ref = oracle_lib.Run(oracle_lib.RunConfig(L=L, R=R, disorder_seed=L, run_seed=7 + R, betas=betas, n_sweeps=S))
    out = []
    for t in range(1, len(betas)):
        ref.step()
        out.append((ref.population(0), ref.energy_hist(t)))
    return out


def gpu_trace(pa, L, R, betas, S):
    run = pa.Run(L, R, L, 7 + R, betas, n_sweeps=S)
    out = []
    for t in range(1, len(betas)):
        assert run.step() == 0
        out.append((run.population(0), run.energy_hist(t)))
    run.close()
    return out


def assert_same(a, b, ctx):
    for t, ((pa_, ha), (pb, hb)) in enumerate(zip(a, b), start=1):
        for x, y, what in zip(pa_, pb, ("spins", "labels", "energies")):
            assert np.array_equal(x, y), f"{ctx} t={t}: {what}"
        assert np.array_equal(ha, hb), f"{ctx} t={t}: energy histogram"


@pytest.mark.parametrize("L,R", SIZES)
def test_every_shape_matches_the_oracle(pa, oracle_lib, L, R):
    betas = np.array([0.0, 0.7, 1.4])
    ref = oracle_trace(oracle_lib, L, R, betas, 2)
    shapes = pa.sweep_shapes(L)
    assert len(shapes) >= 1
    for i, sh in enumerate(shapes):
        pa.sweep_select(L, i)
        assert pa.sweep_selected(L) == i
        assert_same(gpu_trace(pa, L, R, betas, 2), ref, f"L={L} shape {i} {sh}")
    pa.sweep_select(L, -1)
    assert pa.sweep_selected(L) == 0


def test_autotune_selects_a_shape_and_keeps_results(pa, oracle_lib):
    L, R = 8, 20000
    best, ms = pa.sweep_autotune(L, R, launches=2)
    assert 0 <= best < len(pa.sweep_shapes(L))
    assert pa.sweep_selected(L) == best
    assert all(m > 0 for m in ms)          # every shape fits a GB300
    assert ms[best] == min(ms)
    betas = np.array([0.0, 1.0, 2.0])
    assert_same(gpu_trace(pa, L, 1100, betas, 2), oracle_trace(oracle_lib, L, 1100, betas, 2), "autotuned")
    pa.sweep_select(L, -1)


def test_select_rejects_bad_indices(pa):
    n = len(pa.sweep_shapes(10))
    for bad in (n, -2):
        with pytest.raises(pa.PAError) as e:
            pa.sweep_select(10, bad)
        assert e.value.status == pa.PA_ERR_INVALID
    with pytest.raises(pa.PAError):
        pa.sweep_select(11, 0)
