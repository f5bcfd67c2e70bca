"""CPU oracle for population annealing — TEST INFRASTRUCTURE ONLY.

This package wraps ``pa_oracle.c``, a plain, slow C implementation of population
annealing written step by step from Amey & Machta, "Analysis and Optimization of
Population Annealing" (§II, §III.C, §IV.B).  Only the test suite, the smoke check
and the benchmark's CPU-baseline leg may import it; the CUDA library never does,
and the two share no code.

``build()`` compiles ``liboracle.so`` next to this file with gcc (OpenMP over
replica slots, ``-ffp-contract=off`` so floating point rounds as written).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_SRC_GAUSS = os.path.join(_HERE, "pa_oracle_gauss.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, DONE, ERR_INVALID, ERR_NOMEM, ERR_CAPACITY = 0, 1, -1, -2, -3
P_COUPLINGS, P_INIT, P_METROPOLIS, P_RESAMPLE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (returns its path)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_GAUSS),
                                               os.path.getmtime(os.path.join(_HERE, "pa_oracle.h")))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, _SRC_GAUSS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Config(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32),
        ("R", ctypes.c_int64),
        ("R_cap", ctypes.c_int64),
        ("disorder_seed", ctypes.c_uint64),
        ("run_seed", ctypes.c_uint64),
        ("n_pop", ctypes.c_int32),
        ("n_temps", ctypes.c_int32),
        ("betas", ctypes.POINTER(ctypes.c_double)),
        ("beta_max", ctypes.c_double),
        ("eps_target", ctypes.c_double),
        ("n_sweeps", ctypes.c_int32),
        ("sweeps_per_step", ctypes.POINTER(ctypes.c_int32)),
        ("q_bins", ctypes.c_int32),
        ("n_threads", ctypes.c_int32),
    ]


class Obs(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_int32),
        ("beta", ctypes.c_double),
        ("dbeta", ctypes.c_double),
        ("R_tilde", ctypes.c_int64),
        ("sum_E", ctypes.c_int64),
        ("sum_E2", ctypes.c_int64),
        ("E_min", ctypes.c_int32),
        ("mean_E", ctypes.c_double),
        ("var_E", ctypes.c_double),
        ("kmin_prev", ctypes.c_int32),
        ("S_prime", ctypes.c_double),
        ("lnQ", ctypes.c_double),
        ("minus_beta_F", ctypes.c_double),
        ("eps_expected", ctypes.c_double),
        ("culled", ctypes.c_int64),
        ("sum_eta2", ctypes.c_int64),
        ("n_families", ctypes.c_int64),
        ("rho_t", ctypes.c_double),
        ("S_f", ctypes.c_double),
        ("rho_s", ctypes.c_double),
        ("E0", ctypes.c_int32),
        ("g0_tilde", ctypes.c_double),
        ("g0_bar", ctypes.c_double),
        ("q_pairs", ctypes.c_int64),
        ("q_abs_le_02", ctypes.c_int64),
        ("I02", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


class GObs(ctypes.Structure):
    """Observables of a Gaussian-coupling run (org_obs)."""
    _fields_ = [
        ("t", ctypes.c_int32), ("beta", ctypes.c_double), ("dbeta", ctypes.c_double),
        ("R_tilde", ctypes.c_int64), ("sum_E", ctypes.c_int64), ("sum_E2", ctypes.c_double),
        ("E_min", ctypes.c_int64), ("mean_E", ctypes.c_double), ("var_E", ctypes.c_double),
        ("E_min_prev", ctypes.c_int64), ("S_prime", ctypes.c_double), ("lnQ", ctypes.c_double),
        ("minus_beta_F", ctypes.c_double), ("eps_expected", ctypes.c_double), ("culled", ctypes.c_int64),
        ("sum_eta2", ctypes.c_int64), ("n_families", ctypes.c_int64), ("rho_t", ctypes.c_double),
        ("S_f", ctypes.c_double), ("rho_s", ctypes.c_double), ("E0", ctypes.c_int64),
        ("g0_tilde", ctypes.c_double), ("g0_bar", ctypes.c_double), ("q_pairs", ctypes.c_int64),
        ("q_abs_le_02", ctypes.c_int64), ("I02", ctypes.c_double), ("ql_sum", ctypes.c_int64),
        ("ql_mean", ctypes.c_double), ("e_l", ctypes.c_double), ("delta_KY", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i8p = ctypes.POINTER(ctypes.c_int8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        sig = {
            "or_philox4x32_10": (None, [u32p, u32p, u32p]),
            "or_key": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, u32p]),
            "or_couplings": (None, [ctypes.c_int32, ctypes.c_uint64, i8p]),
            "or_energy": (ctypes.c_int32, [ctypes.c_int32, i8p, i8p]),
            "or_metropolis_thresholds": (None, [ctypes.c_double, u32p]),
            "or_metropolis_uniform": (ctypes.c_uint32, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32,
                                                         ctypes.c_uint32, ctypes.c_int64, ctypes.c_int32]),
            "or_metropolis_test": (ctypes.c_int32, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                                    ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32]),
            "or_sweep_replica": (ctypes.c_int32, [ctypes.c_int32, i8p, i8p, ctypes.c_uint64, ctypes.c_int32,
                                                  ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, u32p]),
            "or_reweight": (ctypes.c_int32, [ctypes.c_int32, i64p, ctypes.c_int64, ctypes.c_double, dp,
                                             i32p, u32p, dp]),
            "or_copy_count": (ctypes.c_int32, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                               ctypes.c_int32, ctypes.c_uint32]),
            "or_copy_counts": (None, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, i32p, i32p,
                                      u32p, i32p]),
            "or_resample_uniforms": (None, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, u32p]),
            "or_resample_tau": (None, [ctypes.c_int64, dp, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, i32p]),
            "or_enumerate_levels": (ctypes.c_int, [ctypes.c_int32, i8p, i64p]),
            "or_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(vp)]),
            "or_step": (ctypes.c_int, [vp]),
            "or_run_all": (ctypes.c_int, [vp]),
            "or_current_step": (ctypes.c_int32, [vp]),
            "or_observables": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Obs)]),
            "or_energy_hist": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32, i64p]),
            "or_family_hist": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int64, i64p, i64p, i64p]),
            "or_q_hist": (ctypes.c_int, [vp, ctypes.c_int32, i64p]),
            "or_population": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int64, i8p, i32p, i32p, i64p]),
            "or_last_counts": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int64, i32p, i64p]),
            "or_couplings_of": (i8p, [vp]),
            "or_beta": (ctypes.c_double, [vp, ctypes.c_int32]),
            "or_destroy": (None, [vp]),
            "org_couplings": (None, [ctypes.c_int32, ctypes.c_uint64, i32p]),
            "org_energy": (ctypes.c_int64, [ctypes.c_int32, i32p, i8p]),
            "org_acceptance_threshold": (ctypes.c_uint32, [ctypes.c_double, ctypes.c_int64]),
            "org_metropolis_uniform": (ctypes.c_uint32, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                                          ctypes.c_int32]),
            "org_sweep_replica": (ctypes.c_int64, [ctypes.c_int32, i32p, i8p, ctypes.c_uint64, ctypes.c_int32,
                                                   ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double]),
            "org_weight": (ctypes.c_double, [ctypes.c_double, ctypes.c_int64]),
            "org_reweight": (ctypes.c_int, [i64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, i64p, dp, dp,
                                            dp]),
            "org_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(vp)]),
            "org_step": (ctypes.c_int, [vp]),
            "org_run_all": (ctypes.c_int, [vp]),
            "org_current_step": (ctypes.c_int32, [vp]),
            "org_observables": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(GObs)]),
            "org_q_hist": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32, i64p]),
            "org_population": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int64, i8p, i32p, i64p, i64p]),
            "org_last_counts": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int64, i32p, i64p]),
            "org_couplings_of": (i32p, [vp]),
            "org_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# ---------------------------------------------------------------- building blocks

def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def key(seed: int, purpose: int, pop: int = 0) -> np.ndarray:
    out = np.zeros(2, dtype=np.uint32)
    lib().or_key(seed, purpose, pop, _p(out, ctypes.c_uint32))
    return out


def couplings(L: int, seed: int) -> np.ndarray:
    J = np.zeros(3 * L ** 3, dtype=np.int8)
    lib().or_couplings(L, seed, _p(J, ctypes.c_int8))
    return J


def energy(L: int, J: np.ndarray, s: np.ndarray) -> int:
    J = np.ascontiguousarray(J, dtype=np.int8)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(lib().or_energy(L, _p(J, ctypes.c_int8), _p(s, ctypes.c_int8)))


def metropolis_thresholds(beta: float) -> np.ndarray:
    out = np.zeros(3, dtype=np.uint32)
    lib().or_metropolis_thresholds(beta, _p(out, ctypes.c_uint32))
    return out


def metropolis_uniform(run_seed: int, pop: int, site_index: int, half_sweep: int, slot: int, t: int) -> int:
    """The replica's 32-bit Metropolis uniform: its bit column in the stream (§II)."""
    return int(lib().or_metropolis_uniform(run_seed, pop, site_index, half_sweep, slot, t))


def metropolis_test(run_seed: int, pop: int, site_index: int, half_sweep: int, slot: int, t: int, thr: int) -> bool:
    """uniform < thr, read from the top bit down until the first differing bit."""
    return bool(lib().or_metropolis_test(run_seed, pop, site_index, half_sweep, slot, t, thr))


def sweep_replica(L: int, J: np.ndarray, s: np.ndarray, run_seed: int, pop: int, slot: int, t: int,
                  n_sweeps: int, thr: np.ndarray):
    """Run n_sweeps sweeps of one replica; returns (new spins, energy change)."""
    J = np.ascontiguousarray(J, dtype=np.int8)
    s2 = np.array(s, dtype=np.int8, copy=True)
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    dE = lib().or_sweep_replica(L, _p(J, ctypes.c_int8), _p(s2, ctypes.c_int8), run_seed, pop, slot, t,
                                n_sweeps, _p(thr, ctypes.c_uint32))
    return s2, int(dE)


def reweight(c: np.ndarray, R: int, dbeta: float):
    """Returns (kmin, S', fl[levels], thr[levels], eps_expected)."""
    c = np.ascontiguousarray(c, dtype=np.int64)
    n = c.shape[0]
    fl = np.zeros(n, dtype=np.int32)
    thr = np.zeros(n, dtype=np.uint32)
    S = ctypes.c_double()
    eps = ctypes.c_double()
    kmin = lib().or_reweight(n, _p(c, ctypes.c_int64), R, dbeta, ctypes.byref(S), _p(fl, ctypes.c_int32),
                             _p(thr, ctypes.c_uint32), ctypes.byref(eps))
    return int(kmin), S.value, fl, thr, eps.value


def copy_count(run_seed: int, pop: int, t: int, i: int, fl: int, thr: int) -> int:
    return int(lib().or_copy_count(run_seed, pop, t, i, fl, thr))


def resample_tau(tau: np.ndarray, seed: int, t: int, pop: int = 0) -> np.ndarray:
    """Copy numbers by the nearest-integer rule for the given tau of old slots 0..n-1."""
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    out = np.zeros(tau.shape[0], dtype=np.int32)
    lib().or_resample_tau(tau.shape[0], _p(tau, ctypes.c_double), seed, pop, t, _p(out, ctypes.c_int32))
    return out


def copy_counts(seed: int, pop: int, t: int, levels: np.ndarray, fl: np.ndarray, thr: np.ndarray) -> np.ndarray:
    """Copy numbers of old slots 0..n-1 at energy levels `levels` from per-level floor/fraction tables."""
    levels = np.ascontiguousarray(levels, dtype=np.int32)
    fl = np.ascontiguousarray(fl, dtype=np.int32)
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    assert levels.size == 0 or (levels.min() >= 0 and levels.max() < fl.size == thr.size)
    out = np.zeros(levels.shape[0], dtype=np.int32)
    lib().or_copy_counts(seed, pop, t, levels.shape[0], _p(levels, ctypes.c_int32), _p(fl, ctypes.c_int32),
                         _p(thr, ctypes.c_uint32), _p(out, ctypes.c_int32))
    return out


def resample_uniforms(seed: int, t: int, n: int, pop: int = 0) -> np.ndarray:
    """The uniform words the resampling at step t draws for old slots 0..n-1."""
    out = np.zeros(n, dtype=np.uint32)
    lib().or_resample_uniforms(seed, pop, t, n, _p(out, ctypes.c_uint32))
    return out


def enumerate_levels(L: int, J: np.ndarray) -> np.ndarray:
    J = np.ascontiguousarray(J, dtype=np.int8)
    g = np.zeros(3 * L ** 3 + 1, dtype=np.int64)
    rc = lib().or_enumerate_levels(L, _p(J, ctypes.c_int8), _p(g, ctypes.c_int64))
    if rc != OK:
        raise RuntimeError(f"or_enumerate_levels failed: {rc}")
    return g


# ---------------------------------------------------------------- full runs

@dataclass
class RunConfig:
    L: int
    R: int
    disorder_seed: int
    run_seed: int
    betas: Optional[np.ndarray] = None      # explicit schedule, or None for adaptive
    n_temps: int = 0                        # adaptive: step limit
    beta_max: float = 0.0
    eps_target: float = 0.0
    n_sweeps: int = 10
    sweeps_per_step: Optional[np.ndarray] = None
    n_pop: int = 1
    q_bins: int = 65
    R_cap: int = 0
    n_threads: int = 0


def default_capacity(R: int) -> int:
    return int(R + 10 * int(np.ceil(np.sqrt(R))) + 1024)


class Run:
    """One oracle PA run (owns the C object)."""

    def __init__(self, cfg: RunConfig):
        self.cfg = cfg
        self.L = cfg.L
        self.N = cfg.L ** 3
        self.n_levels = 3 * self.N + 1
        self._betas = None if cfg.betas is None else np.ascontiguousarray(cfg.betas, dtype=np.float64)
        self._sweeps = (None if cfg.sweeps_per_step is None
                        else np.ascontiguousarray(cfg.sweeps_per_step, dtype=np.int32))
        n_temps = len(self._betas) if self._betas is not None else cfg.n_temps
        c = Config()
        c.L = cfg.L
        c.R = cfg.R
        c.R_cap = cfg.R_cap or default_capacity(cfg.R)
        c.disorder_seed = cfg.disorder_seed
        c.run_seed = cfg.run_seed
        c.n_pop = cfg.n_pop
        c.n_temps = n_temps
        c.betas = _p(self._betas, ctypes.c_double) if self._betas is not None else None
        c.beta_max = cfg.beta_max
        c.eps_target = cfg.eps_target
        c.n_sweeps = cfg.n_sweeps
        c.sweeps_per_step = _p(self._sweeps, ctypes.c_int32) if self._sweeps is not None else None
        c.q_bins = cfg.q_bins
        c.n_threads = cfg.n_threads
        self.R_cap = c.R_cap
        self.n_temps = n_temps
        h = ctypes.c_void_p()
        rc = lib().or_create(ctypes.byref(c), ctypes.byref(h))
        if rc != OK:
            raise RuntimeError(f"or_create failed: {rc}")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().or_destroy(h)
            self._h = None

    def step(self) -> int:
        rc = lib().or_step(self._h)
        if rc < 0:
            raise RuntimeError(f"or_step failed: {rc}")
        return rc

    def run(self) -> None:
        rc = lib().or_run_all(self._h)
        if rc != OK:
            raise RuntimeError(f"or_run_all failed: {rc}")

    @property
    def t(self) -> int:
        return int(lib().or_current_step(self._h))

    def beta(self, t: int) -> float:
        return float(lib().or_beta(self._h, t))

    def obs(self, t: int, pop: int = 0) -> dict:
        o = Obs()
        rc = lib().or_observables(self._h, t, pop, ctypes.byref(o))
        if rc != OK:
            raise RuntimeError(f"or_observables failed: {rc}")
        return o.as_dict()

    def energy_hist(self, t: int, pop: int = 0) -> np.ndarray:
        out = np.zeros(self.n_levels, dtype=np.int64)
        rc = lib().or_energy_hist(self._h, t, pop, _p(out, ctypes.c_int64))
        if rc != OK:
            raise RuntimeError(f"or_energy_hist failed: {rc}")
        return out

    def q_hist(self, t: int) -> np.ndarray:
        out = np.zeros(self.cfg.q_bins, dtype=np.int64)
        rc = lib().or_q_hist(self._h, t, _p(out, ctypes.c_int64))
        if rc != OK:
            raise RuntimeError(f"or_q_hist failed: {rc}")
        return out

    def family_hist(self, pop: int = 0):
        cap = self.R_cap + 1
        eta = np.zeros(cap, dtype=np.int64)
        m = np.zeros(cap, dtype=np.int64)
        n = ctypes.c_int64()
        rc = lib().or_family_hist(self._h, pop, cap, _p(eta, ctypes.c_int64), _p(m, ctypes.c_int64),
                                  ctypes.byref(n))
        if rc != OK:
            raise RuntimeError(f"or_family_hist failed: {rc}")
        return eta[:n.value].copy(), m[:n.value].copy()

    def population(self, pop: int = 0):
        """(spins [R~, N] int8, labels int32, energies int32)."""
        cap = self.R_cap
        s = np.zeros((cap, self.N), dtype=np.int8)
        lab = np.zeros(cap, dtype=np.int32)
        E = np.zeros(cap, dtype=np.int32)
        n = ctypes.c_int64()
        rc = lib().or_population(self._h, pop, cap, _p(s, ctypes.c_int8), _p(lab, ctypes.c_int32),
                                 _p(E, ctypes.c_int32), ctypes.byref(n))
        if rc != OK:
            raise RuntimeError(f"or_population failed: {rc}")
        k = n.value
        return s[:k].copy(), lab[:k].copy(), E[:k].copy()

    def last_counts(self, pop: int = 0) -> np.ndarray:
        out = np.zeros(self.R_cap, dtype=np.int32)
        n = ctypes.c_int64()
        rc = lib().or_last_counts(self._h, pop, self.R_cap, _p(out, ctypes.c_int32), ctypes.byref(n))
        if rc != OK:
            raise RuntimeError(f"or_last_counts failed: {rc}")
        return out[:n.value].copy()

    def couplings(self) -> np.ndarray:
        p = lib().or_couplings_of(self._h)
        return np.ctypeslib.as_array(p, shape=(3 * self.N,)).copy()


# ---------------------------------------------------------------- Gaussian couplings

JSCALE = 2 ** 20


def gcouplings(L: int, seed: int) -> np.ndarray:
    """Fixed-point Gaussian couplings Jq[3N] (units of 2^-20)."""
    J = np.zeros(3 * L ** 3, dtype=np.int32)
    lib().org_couplings(L, seed, _p(J, ctypes.c_int32))
    return J


def genergy(L: int, Jq: np.ndarray, s: np.ndarray) -> int:
    Jq = np.ascontiguousarray(Jq, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(lib().org_energy(L, _p(Jq, ctypes.c_int32), _p(s, ctypes.c_int8)))


def gsweep_replica(L: int, Jq: np.ndarray, s: np.ndarray, run_seed: int, pop: int, slot: int, t: int,
                   n_sweeps: int, beta: float):
    """Sweeps of one replica with Gaussian couplings; returns (new spins, energy change)."""
    Jq = np.ascontiguousarray(Jq, dtype=np.int32)
    s2 = np.array(s, dtype=np.int8, copy=True)
    dE = lib().org_sweep_replica(L, _p(Jq, ctypes.c_int32), _p(s2, ctypes.c_int8), run_seed, pop, slot, t,
                                 n_sweeps, beta)
    return s2, int(dE)


def gmetropolis_uniform(run_seed: int, pop: int, n: int, sweep: int, colour: int, slot: int, t: int) -> int:
    """The 32-bit Metropolis uniform of a replica (Gaussian couplings): upper 16 bits
    from one Philox stream, lower 16 bits from a second one (org_metropolis_uniform)."""
    return int(lib().org_metropolis_uniform(run_seed, pop, n, sweep, colour, slot, t))


def gacceptance_threshold(beta: float, dE: int) -> int:
    """Metropolis threshold of a flip costing dE > 0 (units of 2^-20), Gaussian couplings."""
    return int(lib().org_acceptance_threshold(beta, dE))


def gweight(dbeta: float, d: int) -> float:
    """Resampling weight exp(-dbeta d 2^-20) of a replica d above the lowest energy (Eq. Q)."""
    return float(lib().org_weight(dbeta, int(d)))


def greweight(E: np.ndarray, R: int, dbeta: float):
    """Reweighting of Gaussian-coupling energies E (units of 2^-20) by dbeta, Eqs. (tau),
    (Q), (eq_num_elim): returns (E_min, S', expected culling fraction, tau per replica)."""
    E = np.ascontiguousarray(E, dtype=np.int64)
    tau = np.zeros(E.shape[0], dtype=np.float64)
    Emin, S, eps = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    rc = lib().org_reweight(_p(E, ctypes.c_int64), E.shape[0], R, dbeta, ctypes.byref(Emin), ctypes.byref(S),
                            ctypes.byref(eps), _p(tau, ctypes.c_double))
    if rc != OK:
        raise RuntimeError(f"org_reweight failed: {rc}")
    return int(Emin.value), float(S.value), float(eps.value), tau


class GRun:
    """One oracle PA run with Gaussian couplings (explicit or adaptive schedule)."""

    def __init__(self, cfg: RunConfig):
        self.cfg = cfg
        self.L, self.N = cfg.L, cfg.L ** 3
        self._betas = None if cfg.betas is None else np.ascontiguousarray(cfg.betas, dtype=np.float64)
        self._sweeps = (None if cfg.sweeps_per_step is None
                        else np.ascontiguousarray(cfg.sweeps_per_step, dtype=np.int32))
        c = Config()
        c.L, c.R = cfg.L, cfg.R
        c.R_cap = cfg.R_cap or default_capacity(cfg.R)
        c.disorder_seed, c.run_seed = cfg.disorder_seed, cfg.run_seed
        c.n_pop, c.n_temps = cfg.n_pop, (len(self._betas) if self._betas is not None else cfg.n_temps)
        c.betas = _p(self._betas, ctypes.c_double) if self._betas is not None else None
        c.beta_max, c.eps_target = cfg.beta_max, cfg.eps_target
        c.n_sweeps = cfg.n_sweeps
        c.sweeps_per_step = _p(self._sweeps, ctypes.c_int32) if self._sweeps is not None else None
        c.q_bins, c.n_threads = cfg.q_bins, cfg.n_threads
        self.R_cap, self.n_temps, self.n_pop, self.q_bins = c.R_cap, c.n_temps, cfg.n_pop, cfg.q_bins
        h = ctypes.c_void_p()
        rc = lib().org_create(ctypes.byref(c), ctypes.byref(h))
        if rc != OK:
            raise RuntimeError(f"org_create failed: {rc}")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().org_destroy(h)
            self._h = None

    def step(self) -> int:
        rc = lib().org_step(self._h)
        if rc < 0:
            raise RuntimeError(f"org_step failed: {rc}")
        return rc

    def run(self) -> None:
        rc = lib().org_run_all(self._h)
        if rc != OK:
            raise RuntimeError(f"org_run_all failed: {rc}")

    @property
    def t(self) -> int:
        return int(lib().org_current_step(self._h))

    def obs(self, t: int, pop: int = 0) -> dict:
        o = GObs()
        rc = lib().org_observables(self._h, t, pop, ctypes.byref(o))
        if rc != OK:
            raise RuntimeError(f"org_observables failed: {rc}")
        return o.as_dict()

    def q_hist(self, t: int, link: bool = False) -> np.ndarray:
        out = np.zeros(self.q_bins, dtype=np.int64)
        rc = lib().org_q_hist(self._h, t, int(link), _p(out, ctypes.c_int64))
        if rc != OK:
            raise RuntimeError(f"org_q_hist failed: {rc}")
        return out

    def population(self, pop: int = 0):
        """(spins [R~, N] int8, labels int32, energies int64 in units of 2^-20)."""
        s = np.zeros((self.R_cap, self.N), dtype=np.int8)
        lab = np.zeros(self.R_cap, dtype=np.int32)
        E = np.zeros(self.R_cap, dtype=np.int64)
        n = ctypes.c_int64()
        rc = lib().org_population(self._h, pop, self.R_cap, _p(s, ctypes.c_int8), _p(lab, ctypes.c_int32),
                                  _p(E, ctypes.c_int64), ctypes.byref(n))
        if rc != OK:
            raise RuntimeError(f"org_population failed: {rc}")
        k = n.value
        return s[:k].copy(), lab[:k].copy(), E[:k].copy()

    def last_counts(self, pop: int = 0) -> np.ndarray:
        out = np.zeros(self.R_cap, dtype=np.int32)
        n = ctypes.c_int64()
        rc = lib().org_last_counts(self._h, pop, self.R_cap, _p(out, ctypes.c_int32), ctypes.byref(n))
        if rc != OK:
            raise RuntimeError(f"org_last_counts failed: {rc}")
        return out[:n.value].copy()

    def couplings(self) -> np.ndarray:
        p = lib().org_couplings_of(self._h)
        return np.ctypeslib.as_array(p, shape=(3 * self.N,)).copy()
