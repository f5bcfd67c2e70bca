"""Seeded synthetic workloads for population annealing runs.

This module only states input recipes — lattice size, population size, seeds,
temperature schedules and the mixes of batched and served requests.  It holds
none of the method's arithmetic, and both the CUDA path and the CPU oracle take
their inputs from it.

The paper studies the 3D Edwards-Anderson spin glass; its inputs are generated
from seeds (couplings and initial spins), so no dataset is involved.  The
couplings here are +-1 with p = 1/2 (the paper's model draws them from a
Gaussian).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np


def linear_betas(n_temps: int, beta_max: float) -> np.ndarray:
    """beta_t = t * beta_max / (n_temps - 1), t = 0 .. n_temps-1 (beta_0 = 0)."""
    return np.array([t * beta_max / (n_temps - 1) for t in range(n_temps)], dtype=np.float64)


def default_capacity(R: int) -> int:
    """Population capacity R + 10 sqrt(R) + 1024 (the population fluctuates by O(sqrt R))."""
    return int(R + 10 * int(math.ceil(math.sqrt(R))) + 1024)


@dataclass
class Workload:
    name: str
    L: int
    R: int
    disorder_seed: int
    run_seed: int
    betas: Optional[np.ndarray] = None   # explicit schedule; None = adaptive
    n_temps: int = 0                     # adaptive: step limit
    beta_max: float = 5.0
    eps_target: float = 0.0
    n_sweeps: int = 10
    sweeps_per_step: Optional[np.ndarray] = None  # explicit schedule: sweeps of every step (overrides n_sweeps)
    n_pop: int = 1
    q_bins: int = 65
    R_cap: int = 0
    model: int = 0                       # 0: +-1 couplings, 1: Gaussian couplings (explicit schedules)

    @property
    def N(self) -> int:
        return self.L ** 3

    @property
    def capacity(self) -> int:
        return self.R_cap or default_capacity(self.R)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# Plain PA, L=4, seed 1, R=1000, 51 linear temperatures to beta=5, 10 sweeps.
C1 = Workload("L4_R1e3_linear51", L=4, R=1000, disorder_seed=1, run_seed=1001,
              betas=linear_betas(51, 5.0), n_sweeps=10)

# L=8, seed 2, R=1e5, two populations for the overlap, 201 linear temperatures.
C2 = Workload("L8_R1e5_2pop_linear201", L=8, R=100_000, disorder_seed=2, run_seed=1002,
              betas=linear_betas(201, 5.0), n_sweeps=10, n_pop=2, q_bins=65)

# L=10, seed 3, R=1e6, adaptive schedule holding the culling fraction at 0.272
# (the paper's L=10 value, Table I) up to beta=5.
C3 = Workload("L10_R1e6_adaptive", L=10, R=1_000_000, disorder_seed=3, run_seed=1003,
              betas=None, n_temps=4096, beta_max=5.0, eps_target=0.272, n_sweeps=10)


def batched_mix(n_runs: int = 256, first_seed: int = 100, n_temps: int = 101,
                sizes=(4, 6, 8, 10), r_lo: float = 1e4, r_hi: float = 1e5) -> List[Workload]:
    """Many disorder realizations of mixed sizes: L cycles through ``sizes``,
    R is log-uniform in [r_lo, r_hi] from a seeded numpy generator."""
    rng = np.random.default_rng(first_seed)
    out = []
    for i in range(n_runs):
        seed = first_seed + i
        L = sizes[i % len(sizes)]
        u = rng.random()
        R = int(math.floor(r_lo * (r_hi / r_lo) ** u))
        out.append(Workload(f"batch_{seed}", L=L, R=R, disorder_seed=seed, run_seed=10_000 + seed,
                            betas=linear_betas(n_temps, 5.0), n_sweeps=10))
    return out


def serving_stream(n_requests: int = 2000, first_seed: int = 10_000, arrival_seed: int = 7,
                   sizes=(4, 6, 8, 10, 12), r_lo: float = 1e3, r_hi: float = 2e5,
                   temps=(51, 101, 201)):
    """Requests for the serving loop: (workload, relative arrival time in units of
    the mean inter-arrival gap).  Exponential gaps from a fixed generator."""
    rng = np.random.default_rng(arrival_seed)
    out = []
    clock = 0.0
    for i in range(n_requests):
        seed = first_seed + i
        L = int(rng.choice(sizes))
        R = int(math.floor(r_lo * (r_hi / r_lo) ** rng.random()))
        T = int(rng.choice(temps))
        clock += rng.exponential(1.0)
        out.append((Workload(f"req_{seed}", L=L, R=R, disorder_seed=seed, run_seed=50_000 + seed,
                             betas=linear_betas(T, 5.0), n_sweeps=10), clock))
    return out
