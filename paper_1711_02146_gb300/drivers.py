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
katzgraber_young      Delta_KY(beta) = [e_l - e]_J over Gaussian disorder
                      realizations (Eqs. KY, el), two populations per sample.
schedule_comparison   §V.A: rho_t at beta = 5 under the unoptimized schedule
                      (dbeta = 0.05, 10 sweeps per step) and the optimized one
                      (constant culling fraction, 3/22/1 sweeps by temperature
                      range, §IV.B) at equal sweeps per replica, per disorder
                      realization.
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


# ---------------------------------------------------------------- schedule comparison (§IV.B, §V.A)

def paper_sweep_schedule(betas, low: float = 0.5, high: float = 2.5, hot: int = 3, mid: int = 22,
                         cold: int = 1) -> np.ndarray:
    """§IV.B's ad hoc sweep schedule: `hot` sweeps per step below beta = low, `mid`
    for low <= beta <= high, `cold` above (step 0, at beta = 0, does none)."""
    b = np.asarray(betas, dtype=np.float64)
    s = np.where(b < low, hot, np.where(b <= high, mid, cold)).astype(np.int32)
    s[0] = 0
    return s


def constant_culling_betas(L: int, disorder_seed: int, R: int, eps: float, beta_max: float = 5.0,
                           run_seed: int = 1, n_sweeps: int = 10) -> np.ndarray:
    """The beta schedule of one pilot run that holds the culling fraction at eps
    (§IV.B: chosen on a single disorder realization, then reused)."""
    from .workloads import Workload
    w = Workload("pilot", L=L, R=R, disorder_seed=disorder_seed, run_seed=run_seed, betas=None, n_temps=4096,
                 beta_max=beta_max, eps_target=eps, n_sweeps=n_sweeps)
    run = pa.Run.from_workload(w)
    run.run()
    betas = np.array([run.beta(t) for t in range(run.t + 1)])
    run.close()
    return betas


def matched_optimized_schedule(L: int, disorder_seed: int, R: int, total_sweeps: int, beta_max: float = 5.0,
                               run_seed: int = 1, iters: int = 14):
    """A constant-culling beta schedule with the paper's 3/22/1 sweep schedule whose
    total number of sweeps per replica is as close as bisection on eps gets to
    `total_sweeps` (the comparison of §V.A holds the work fixed).  Returns
    (betas, sweeps_per_step, eps)."""
    lo, hi = 1e-3, 0.9            # larger eps -> bigger steps -> fewer sweeps
    best = None
    for _ in range(iters):
        eps = math.sqrt(lo * hi)
        betas = constant_culling_betas(L, disorder_seed, R, eps, beta_max, run_seed)
        sw = paper_sweep_schedule(betas)
        total = int(sw.sum())
        if best is None or abs(total - total_sweeps) < abs(best[1].sum() - total_sweeps):
            best = (betas, sw, eps)
        if total == total_sweeps:
            break
        if total > total_sweeps:
            lo = eps
        else:
            hi = eps
    return best


def schedule_comparison(L: int, R: int, disorder_seeds, beta_max: float = 5.0, dbeta: float = 0.05,
                        sweeps: int = 10, pilot_R: int = 20000, run_seed: int = 11) -> Dict[str, object]:
    """§V.A: rho_t at beta_max under the unoptimized schedule (constant dbeta,
    `sweeps` sweeps per step) and the optimized one (constant culling fraction,
    3/22/1 sweeps, the same total sweeps per replica), for every disorder
    realization; all 2M runs advance together as one batch."""
    from .workloads import Workload, linear_betas
    n = int(round(beta_max / dbeta)) + 1
    b_un = linear_betas(n, beta_max)
    s_un = np.full(n, sweeps, dtype=np.int32)
    s_un[0] = 0
    seeds = list(disorder_seeds)
    b_op, s_op, eps = matched_optimized_schedule(L, seeds[0], pilot_R, int(s_un.sum()), beta_max)
    ws = []
    for d in seeds:
        ws.append(Workload(f"unopt_{d}", L=L, R=R, disorder_seed=d, run_seed=run_seed, betas=b_un,
                           sweeps_per_step=s_un))
        ws.append(Workload(f"opt_{d}", L=L, R=R, disorder_seed=d, run_seed=run_seed, betas=b_op, sweeps_per_step=s_op))
    batch = pa.Batch(ws)
    batch.run()
    rho = np.zeros((len(seeds), 2))
    for i in range(len(ws)):
        v = batch.run_view(i)
        rho[i // 2, i % 2] = v.obs(v.t)["rho_t"]
    batch.close()
    ratio = rho[:, 0] / rho[:, 1]
    return {"rho_unopt": rho[:, 0], "rho_opt": rho[:, 1], "ratio": ratio,
            "geo_mean_ratio": float(np.exp(np.mean(np.log(ratio)))),
            "ratio_of_means": float(rho[:, 0].mean() / rho[:, 1].mean()),
            "eps": eps, "n_steps_opt": len(b_op), "n_steps_unopt": n,
            "sweeps_opt": int(s_op.sum()), "sweeps_unopt": int(s_un.sum())}


# ---------------------------------------------------------------- Katzgraber-Young measure (§II.A)

def katzgraber_young(L: int, R: int, disorder_seeds, betas, n_sweeps: int = 10, run_seed: int = 1):
    """Delta_KY(beta) = [e_l - e]_J (Eqs. KY, el) over Gaussian disorder
    realizations: every sample runs two independent populations (model 1) as
    one batch; returns per step the disorder averages of e, e_l and their
    difference with its standard error."""
    from .workloads import Workload
    seeds = list(disorder_seeds)
    ws = [Workload(f"ky_{d}", L=L, R=R, disorder_seed=d, run_seed=run_seed, betas=np.asarray(betas, np.float64),
                   n_sweeps=n_sweeps, n_pop=2, model=1) for d in seeds]
    batch = pa.Batch(ws)
    batch.run()
    T = len(betas)
    e = np.zeros((len(seeds), T))
    el = np.zeros((len(seeds), T))
    for i in range(len(ws)):
        v = batch.run_view(i)
        for t in range(T):
            o = v.gobs(t, 0)
            e[i, t] = o["mean_E"] / (L ** 3)
            el[i, t] = o["e_l"]
    batch.close()
    d = el - e
    return {"beta": np.asarray(betas, np.float64), "e": e.mean(axis=0), "e_l": el.mean(axis=0),
            "delta_KY": d.mean(axis=0), "delta_KY_err": d.std(axis=0, ddof=1) / math.sqrt(len(seeds))}
