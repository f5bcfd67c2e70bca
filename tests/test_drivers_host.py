"""Host logic of the paper's procedures (drivers.py) on the CPU: the §IV.B sweep
schedule and the §IV.A population-size rule, with the GPU run replaced by a
stand-in that reports a chosen rho_t (no kernels involved)."""
import numpy as np
import pytest

from paper_1711_02146_gb300 import drivers
from paper_1711_02146_gb300.workloads import Workload, linear_betas


def test_paper_sweep_schedule_by_temperature_range():
    b = linear_betas(101, 5.0)  # beta = 0.05 t
    s = drivers.paper_sweep_schedule(b)
    assert s.dtype == np.int32 and s.shape == b.shape
    assert s[0] == 0                              # step 0 does no sweeps
    for t in range(1, 101):
        beta = 0.05 * t
        want = 3 if beta < 0.5 - 1e-12 else (22 if beta <= 2.5 + 1e-12 else 1)
        assert s[t] == want, (t, beta)
    assert s[10] == 22 and s[50] == 22 and s[51] == 1  # both ends of [0.5, 2.5] take 22


class _FakeRun:
    """Stands in for pa.Run: rho_t at the last step is a function of R."""
    rho_of_R = staticmethod(lambda R: 50.0)
    created = []

    def __init__(self, w):
        self.R = w.R
        self.t = 7
        _FakeRun.created.append(w.R)

    @classmethod
    def from_workload(cls, w):
        assert w.R_cap == 0  # capacity follows the new R
        return cls(w)

    def run(self):
        pass

    def obs(self, t):
        assert t == self.t
        return {"rho_t": float(self.rho_of_R(self.R))}

    def close(self):
        pass


@pytest.fixture
def fake_runs(monkeypatch):
    monkeypatch.setattr(drivers.pa, "Run", _FakeRun)
    _FakeRun.created = []
    yield _FakeRun


def _w():
    return Workload("hap", L=8, R=1000, disorder_seed=1, run_seed=2, betas=linear_betas(11, 5.0))


def test_hardness_adaptive_population_grows_until_equilibrated(fake_runs):
    fake_runs.rho_of_R = staticmethod(lambda R: 50.0)
    res = drivers.hardness_adaptive_population(_w(), R0=200)
    # 200 <= 100 * 50, so rerun with R = 150 * 50 = 7500 > 100 * 50: equilibrated
    assert fake_runs.created == [200, 7500]
    assert res["equilibrated"] and res["R"] == 7500 and res["rho_t"] == 50.0
    assert res["history"] == [(200, 50.0), (7500, 50.0)]


def test_hardness_adaptive_population_accepts_an_equilibrated_first_run(fake_runs):
    fake_runs.rho_of_R = staticmethod(lambda R: 9.99)
    res = drivers.hardness_adaptive_population(_w(), R0=1000)
    assert fake_runs.created == [1000] and res["equilibrated"] and res["R"] == 1000


def test_hardness_adaptive_population_gives_up_after_max_rounds(fake_runs):
    # rho_t proportional to R never satisfies R > 100 rho_t
    fake_runs.rho_of_R = staticmethod(lambda R: R / 50.0)
    res = drivers.hardness_adaptive_population(_w(), R0=100, max_rounds=3)
    assert fake_runs.created == [100, 300, 900]  # R -> ceil(150 * R / 50) = 3 R
    assert not res["equilibrated"] and res["R"] == 900 and len(res["history"]) == 3


def test_hardness_adaptive_population_boundary_is_strict(fake_runs):
    # R = 100 rho_t exactly is not yet equilibrated (the rule asks for R > 100 rho_t)
    fake_runs.rho_of_R = staticmethod(lambda R: R / 100.0)
    res = drivers.hardness_adaptive_population(_w(), R0=500, max_rounds=2)
    assert fake_runs.created == [500, 750] and not res["equilibrated"]


class _FakeView:
    def __init__(self, m, T):
        self.m, self.T = m, T

    def obs(self, t):
        # run m: -beta F = m * t (so the variance over m = 0, 1, 2 is t^2), rho_t = 1 + m,
        # eps = 0.1 at every step but 0 (run-independent)
        return {"minus_beta_F": float(self.m * t), "rho_t": 1.0 + self.m, "eps_expected": 0.0 if t == 0 else 0.1}


class _FakeBatch:
    seeds = []

    def __init__(self, ws):
        _FakeBatch.seeds = [w.run_seed for w in ws]
        self.T = len(ws[0].betas)

    def run(self):
        pass

    def run_view(self, m):
        return _FakeView(m, self.T)

    def close(self):
        pass


def test_free_energy_variance_aggregates_the_runs(monkeypatch):
    monkeypatch.setattr(drivers.pa, "Batch", _FakeBatch)
    w = Workload("fv", L=4, R=1000, disorder_seed=1, run_seed=2, betas=linear_betas(5, 1.0))
    r = drivers.free_energy_variance(w, M=3, first_run_seed=40)
    assert _FakeBatch.seeds == [40, 41, 42]                     # runs differ only in their run seed
    t = np.arange(5)
    assert np.allclose(r["rho_f"], 1000 * t ** 2)               # R var(beta F~), var over m = 0, 1, 2 of m t is t^2
    assert np.allclose(r["rho_f_err"], np.sqrt(2 / 2) * 1000 * t ** 2)
    assert np.allclose(r["rho_t"], 2.0) and np.allclose(r["rho_t_err"], 1 / np.sqrt(3))
    eps = np.where(t == 0, 0.0, 0.1)
    assert np.allclose(r["rho_t_grow"], 1 + 0.2 * t)            # Eq. rhotb with eps = 0.1 from step 1
    assert np.allclose(r["rho_f_grow"], 2 * np.pi * 0.01 * t)   # Eq. rhofgrow
    assert np.allclose(r["rho_f_from_rho_t"], 2.0 - 1.0 - np.cumsum(2 * eps - 2 * np.pi * eps ** 2))
    with pytest.raises(ValueError):
        drivers.free_energy_variance(w, M=1)


class _FakeGView:
    def __init__(self, w):
        self.w = w

    def gobs(self, t, pop):
        assert pop == 0
        d = self.w.disorder_seed
        # sample d: mean energy -N (d + t) (so e = -(d + t)), link energy e_l = -(d + t) + 0.01 d
        return {"mean_E": -float(self.w.N * (d + t)), "e_l": -(d + t) + 0.01 * d}


class _FakeGBatch:
    made = []

    def __init__(self, ws):
        _FakeGBatch.made = list(ws)
        self.ws = ws

    def run(self):
        pass

    def run_view(self, i):
        return _FakeGView(self.ws[i])

    def close(self):
        pass


def test_katzgraber_young_aggregates_over_disorder(monkeypatch):
    monkeypatch.setattr(drivers.pa, "Batch", _FakeGBatch)
    betas = np.linspace(0.0, 1.0, 4)
    r = drivers.katzgraber_young(4, 500, [1, 2, 3], betas, n_sweeps=5, run_seed=9)
    ws = _FakeGBatch.made
    assert [w.disorder_seed for w in ws] == [1, 2, 3]
    assert all(w.n_pop == 2 and w.model == 1 and w.run_seed == 9 and w.n_sweeps == 5 for w in ws)
    t = np.arange(4)
    assert np.allclose(r["e"], -(2 + t))                # disorder mean of e = E / N
    assert np.allclose(r["delta_KY"], 0.02)              # [e_l - e] = mean of 0.01 d over d = 1, 2, 3
    assert np.allclose(r["delta_KY_err"], np.std([0.01, 0.02, 0.03], ddof=1) / np.sqrt(3))
