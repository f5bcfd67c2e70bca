"""Host-side procedures of the paper built on the GPU runs (no kernels here).

free_energy_variance  rho_f from M independent runs of one disorder realization
                      (§III.A Eq. rhof, error bar Eq. gaussian_err), beside the
                      estimates the paper derives from one run's culling
                      fractions and family statistics: rho_f = 2 pi sum eps^2
                      (Eq. rhofgrow), rho_t - 1 = 2 sum eps (Eq. rhotb) and
                      rho_f ~ rho_t - 1 - sum (2 eps - 2 pi eps^2) (Eq. rhofratiorhot).
hardness_adaptive_population
                      the population-size scheme of §IV.A: run with R0; while
                      R <= 100 rho_t(R), rerun with R = 150 rho_t(R).
The M runs of free_energy_variance advance together as one batch (pa_batch).
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

from . import pa


def free_energy_variance(workload, M: int, first_run_seed: int = 1) -> Dict[str, np.ndarray]:
    """Statistics over M runs of `workload` that differ only in their run seed.

    Returns per step t: beta, rho_f = R var(beta F~) over the runs, its error
    sqrt(2/(M-1)) rho_f, the run-averaged rho_t and culling fraction eps, and
    the paper's estimates rho_f_grow = 2 pi sum_{u<=t} eps_u^2,
    rho_t_grow = 1 + 2 sum eps_u and rho_f_from_rho_t = rho_t - 1 - sum (2 eps_u - 2 pi eps_u^2).
    """
    if M < 2:
        raise ValueError("M >= 2 runs are needed for a variance")
    ws = [workload.with_(run_seed=first_run_seed + m, name=f"{workload.name}_m{m}") for m in range(M)]
    batch = pa.Batch(ws)
    batch.run()
    T = len(workload.betas)
    mbf = np.zeros((M, T))
    rho_t = np.zeros((M, T))
    eps = np.zeros((M, T))
    for m in range(M):
        v = batch.run_view(m)
        for t in range(T):
            o = v.obs(t)
            mbf[m, t] = o["minus_beta_F"]
            rho_t[m, t] = o["rho_t"]
            eps[m, t] = o["eps_expected"]
    batch.close()
    rho_f = workload.R * mbf.var(axis=0, ddof=1)
    e = eps.mean(axis=0)
    rt = rho_t.mean(axis=0)
    return {
        "beta": np.asarray(workload.betas, dtype=np.float64),
        "rho_f": rho_f,
        "rho_f_err": math.sqrt(2.0 / (M - 1)) * rho_f,
        "rho_t": rt,
        "rho_t_err": rho_t.std(axis=0, ddof=1) / math.sqrt(M),
        "eps": e,
        "rho_f_grow": 2.0 * math.pi * np.cumsum(e ** 2),
        "rho_t_grow": 1.0 + 2.0 * np.cumsum(e),
        "rho_f_from_rho_t": rt - 1.0 - np.cumsum(2.0 * e - 2.0 * math.pi * e ** 2),
    }


def hardness_adaptive_population(workload, R0: int, check: float = 100.0, grow: float = 150.0,
                                 max_rounds: int = 6) -> Dict[str, object]:
    """§IV.A: run with R0; the run is equilibrated when R > check * rho_t(R) at the
    last step, otherwise rerun with R = grow * rho_t(R).  Returns the final R, its
    rho_t, whether the criterion was met, and the (R, rho_t) history."""
    R = int(R0)
    history: List[tuple] = []
    for _ in range(max_rounds):
        run = pa.Run.from_workload(workload.with_(R=R, R_cap=0))
        run.run()
        rt = run.obs(run.t)["rho_t"]
        run.close()
        history.append((R, rt))
        if R > check * rt:
            return {"R": R, "rho_t": rt, "equilibrated": True, "history": history}
        R = int(math.ceil(grow * rt))
    return {"R": history[-1][0], "rho_t": history[-1][1], "equilibrated": False, "history": history}
