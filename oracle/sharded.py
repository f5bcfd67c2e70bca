"""CPU-rank emulation of a population sharded across P ranks (test infrastructure).

The population of every step is split by slot into P contiguous, balanced blocks
(rank r holds slots [r R~/P, (r+1) R~/P) of every population; with two
populations the blocks are cut from max(R~_A, R~_B) so that slot j of both lives
on the same rank).  One temperature step (§II) then needs, per population:

  1. the energy-level histogram of the previous step: an all-reduce of integer
     counts (exact, so every rank computes the same tau tables, Eq. tau);
  2. the copy numbers of the local old slots (nearest-integer rule; the random
     word of old slot i depends on its global index only);
  3. the global offset of the rank's copies: an all-gather of one total per rank
     and an exclusive scan of those totals;
  4. a point-to-point exchange that moves every copy to the rank owning its new
     slot (each distinct parent travels once, with its multiplicity);
  5. the sweeps of the local new slots (their random words depend on the global
     new slot only);
  6. the measurements: all-reduced histogram and energy sums, the minimum energy,
     family statistics from the runs of sorted labels with a boundary exchange of
     each rank's first and last run (families may straddle ranks), and the local
     overlap histograms of co-located slot pairs, all-reduced.

Every random word is addressed by global slot, so a P-rank run must reproduce
the single-process oracle (oracle.Run) bit for bit; tests/test_sharded_emulation.py
checks that.  Only the building blocks of the oracle (oracle.reweight,
copy_count, sweep_replica, energy, couplings, philox) are used, and the
exchanges go through torch.distributed (gloo on CPU).  Explicit schedules only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import copy_count, couplings, energy, key, metropolis_thresholds, philox, reweight, sweep_replica

P_INIT = 1  # random-stream purpose of the initial spins


def block(R: int, P: int, r: int):
    """Slots [lo, hi) of rank r when R slots are split into P balanced blocks."""
    return (r * R) // P, ((r + 1) * R) // P


@dataclass
class ShardPop:
    lo: int                      # global slot of local slot 0
    R_tilde: int                 # global population size
    s: np.ndarray                # [n_local, N] int8
    lab: np.ndarray              # [n_local] int32 family labels (sorted globally)
    E: np.ndarray                # [n_local] int32 energies
    lnQ_sum: float = 0.0
    E0: int = 0
    hist: List[np.ndarray] = field(default_factory=list)   # global level histogram of every step
    obs: List[dict] = field(default_factory=list)
    counts: Optional[np.ndarray] = None                     # local copy numbers of the last step


class ShardedRun:
    """One rank's part of a sharded population annealing run (explicit schedule)."""

    def __init__(self, L: int, R: int, disorder_seed: int, run_seed: int, betas, n_sweeps: int,
                 n_pop: int = 1, q_bins: int = 65, R_cap: Optional[int] = None):
        import torch.distributed as dist
        self.dist = dist
        self.P, self.rank = dist.get_world_size(), dist.get_rank()
        self.L, self.N, self.R = L, L ** 3, R
        self.n_levels = 3 * self.N + 1
        self.run_seed, self.n_pop, self.q_bins = run_seed, n_pop, q_bins
        self.betas = np.asarray(betas, dtype=np.float64)
        self.n_sweeps = n_sweeps
        self.R_cap = R_cap if R_cap is not None else R + 10 * math.ceil(math.sqrt(R)) + 1024
        self.J = couplings(L, disorder_seed)
        self.t = 0
        self.qhist: List[np.ndarray] = []
        lo, hi = block(R, self.P, self.rank)
        self.pops = [self._initial(p, lo, hi) for p in range(n_pop)]
        self._measure(0)

    # ------------------------------------------------------------ collectives
    def _allreduce(self, a: np.ndarray, op="sum") -> np.ndarray:
        import torch
        x = torch.from_numpy(np.ascontiguousarray(a, dtype=np.int64).copy())
        self.dist.all_reduce(x, op={"sum": self.dist.ReduceOp.SUM, "min": self.dist.ReduceOp.MIN,
                                    "max": self.dist.ReduceOp.MAX}[op])
        return x.numpy()

    def _allgather(self, a: np.ndarray) -> np.ndarray:
        import torch
        x = torch.from_numpy(np.ascontiguousarray(a, dtype=np.int64).copy())
        out = [torch.zeros_like(x) for _ in range(self.P)]
        self.dist.all_gather(out, x)
        return np.stack([o.numpy() for o in out])

    # ------------------------------------------------------------ state
    def _initial(self, p: int, lo: int, hi: int) -> ShardPop:
        k = key(self.run_seed, P_INIT, p)
        n = hi - lo
        s = np.empty((n, self.N), dtype=np.int8)
        for jj in range(n):
            j = lo + jj
            for site in range(self.N):
                w = philox((site, 0, j >> 2, 0), k)[j & 3]
                s[jj, site] = 1 if (w & 1) == 0 else -1
        E = np.array([energy(self.L, self.J, s[jj]) for jj in range(n)], dtype=np.int32)
        return ShardPop(lo=lo, R_tilde=self.R, s=s, lab=np.arange(lo, hi, dtype=np.int32), E=E)

    # ------------------------------------------------------------ one step
    def step(self) -> None:
        t = self.t + 1
        dbeta = float(self.betas[t] - self.betas[t - 1])
        met = metropolis_thresholds(float(self.betas[t]))
        N = self.N
        plans = []
        for p, P_ in enumerate(self.pops):
            kmin, S, fl, thr, eps = reweight(P_.hist[t - 1], self.R, dbeta)
            k = (P_.E.astype(np.int64) + 3 * N) // 2
            cnt = np.array([copy_count(self.run_seed, p, t, P_.lo + i, int(fl[k[i]]), int(thr[k[i]]))
                            for i in range(P_.E.shape[0])], dtype=np.int64)
            totals = self._allgather(np.array([cnt.sum(), (cnt == 0).sum()]))
            offset = int(totals[: self.rank, 0].sum())
            newR = int(totals[:, 0].sum())
            if newR > self.R_cap:
                raise RuntimeError("population outgrew its capacity")
            if newR == 0:
                raise RuntimeError("every replica received zero copies")
            Emin_prev = 2 * kmin - 3 * N
            lnQ = math.log(S / float(P_.R_tilde)) - dbeta * float(Emin_prev)
            plans.append(dict(cnt=cnt, offset=offset, newR=newR, culled=int(totals[:, 1].sum()), kmin=kmin, S=S,
                              eps=eps, lnQ=lnQ))
        R_part = max(pl["newR"] for pl in plans)    # common blocks: slot j of every population co-located
        for p, (P_, pl) in enumerate(zip(self.pops, plans)):
            self._exchange(P_, pl, R_part)
            P_.counts = pl["cnt"].astype(np.int32)
            P_.lnQ_sum = P_.lnQ_sum + pl["lnQ"]
            P_.R_tilde = pl["newR"]
            for jj in range(P_.E.shape[0]):
                s2, dE = sweep_replica(self.L, self.J, P_.s[jj], self.run_seed, p, P_.lo + jj, t, self.n_sweeps, met)
                P_.s[jj] = s2
                P_.E[jj] += dE
            P_.obs.append(None)   # filled by _measure
            P_._step_fields = dict(dbeta=dbeta, kmin_prev=pl["kmin"], S_prime=pl["S"], lnQ=pl["lnQ"],
                                   eps_expected=pl["eps"], culled=pl["culled"])
        self.t = t
        self._measure(t)

    def _exchange(self, P_: ShardPop, pl: dict, R_part: int) -> None:
        """Moves every copy to the rank that owns its new slot (point to point)."""
        import torch
        dist = self.dist
        cnt = pl["cnt"]
        first = pl["offset"] + np.concatenate([[0], np.cumsum(cnt)[:-1]]) if cnt.size else np.zeros(0, np.int64)
        sends = {}
        for q in range(self.P):
            lo_q, hi_q = block(R_part, self.P, q)
            hi_q = min(hi_q, pl["newR"])
            lo_q = min(lo_q, hi_q)
            m = np.clip(np.minimum(first + cnt, hi_q) - np.maximum(first, lo_q), 0, None)
            idx = np.nonzero(m)[0]
            sends[q] = (idx, m[idx])
        reqs, keep = [], []
        for q in range(self.P):
            if q == self.rank:
                continue
            idx, m = sends[q]
            hdr = torch.tensor([idx.size], dtype=torch.int64)
            keep.append(hdr)
            reqs.append(dist.isend(hdr, q))
            if idx.size:
                for arr in (P_.s[idx].reshape(-1), P_.lab[idx], P_.E[idx], m.astype(np.int32)):
                    ten = torch.from_numpy(np.ascontiguousarray(arr).copy())
                    keep.append(ten)
                    reqs.append(dist.isend(ten, q))
        parts = []
        for src in range(self.P):    # sources in rank order = new slots in global order
            if src == self.rank:
                idx, m = sends[src]
                parts.append((P_.s[idx], P_.lab[idx], P_.E[idx], m))
                continue
            hdr = torch.zeros(1, dtype=torch.int64)
            dist.recv(hdr, src)
            n = int(hdr.item())
            if n == 0:
                continue
            s = torch.zeros(n * self.N, dtype=torch.int8)
            lab = torch.zeros(n, dtype=torch.int32)
            E = torch.zeros(n, dtype=torch.int32)
            m = torch.zeros(n, dtype=torch.int32)
            for ten in (s, lab, E, m):
                dist.recv(ten, src)
            parts.append((s.numpy().reshape(n, self.N), lab.numpy(), E.numpy(), m.numpy()))
        for rq in reqs:
            rq.wait()
        if parts:
            rep = np.concatenate([np.asarray(pp[3], dtype=np.int64) for pp in parts])
            P_.s = np.repeat(np.concatenate([pp[0] for pp in parts]), rep, axis=0)
            P_.lab = np.repeat(np.concatenate([pp[1] for pp in parts]), rep).astype(np.int32)
            P_.E = np.repeat(np.concatenate([pp[2] for pp in parts]), rep).astype(np.int32)
        else:
            P_.s = np.zeros((0, self.N), dtype=np.int8)
            P_.lab = np.zeros(0, dtype=np.int32)
            P_.E = np.zeros(0, dtype=np.int32)
        lo_r, _ = block(R_part, self.P, self.rank)
        P_.lo = min(lo_r, pl["newR"])

    # ------------------------------------------------------------ measurement
    def _families(self, P_: ShardPop):
        """sum eta^2, number of families and the size histogram m(eta): local runs
        of sorted labels, with the first and last run of every rank joined across
        rank boundaries (a family may span several ranks)."""
        lab = P_.lab
        if lab.size:
            change = np.nonzero(lab[1:] != lab[:-1])[0] + 1
            starts = np.concatenate([[0], change])
            lens = np.diff(np.concatenate([starts, [lab.size]]))
            runs = lab[starts]
            info = [1, runs[0], lens[0], runs[-1], lens[-1], lens.size]
            interior = lens[1:-1] if lens.size > 2 else np.zeros(0, dtype=np.int64)
        else:
            info = [0, 0, 0, 0, 0, 0]
            interior = np.zeros(0, dtype=np.int64)
        edges = self._allgather(np.array(info))
        joined, open_lab, open_len = [], None, 0
        for has, f, lf, l, ll, nr in edges:
            if not has:
                continue
            if nr == 1:
                if open_lab is not None and f == open_lab:
                    open_len += lf
                else:
                    if open_lab is not None:
                        joined.append(open_len)
                    open_lab, open_len = f, lf
                continue
            if open_lab is not None and f == open_lab:
                joined.append(open_len + lf)
            else:
                if open_lab is not None:
                    joined.append(open_len)
                joined.append(lf)
            open_lab, open_len = l, ll
        if open_lab is not None:
            joined.append(open_len)
        joined = np.asarray(joined, dtype=np.int64)
        sums = self._allreduce(np.array([(interior.astype(np.int64) ** 2).sum(), interior.size]))
        sum_eta2 = int(sums[0] + (joined ** 2).sum())
        n_fam = int(sums[1] + joined.size)
        top = int(self._allreduce(np.array([interior.max() if interior.size else 0]), "max")[0])
        top = max(top, int(joined.max()) if joined.size else 0)
        m = self._allreduce(np.bincount(interior, minlength=top + 1)[: top + 1]) + np.bincount(joined, minlength=top + 1)
        return sum_eta2, n_fam, m

    def _measure(self, t: int) -> None:
        N = self.N
        for p, P_ in enumerate(self.pops):
            k = (P_.E.astype(np.int64) + 3 * N) // 2
            c = self._allreduce(np.bincount(k, minlength=self.n_levels))
            sums = self._allreduce(np.array([P_.E.astype(np.int64).sum(), (P_.E.astype(np.int64) ** 2).sum()]))
            Emin = int(self._allreduce(np.array([P_.E.min() if P_.E.size else 3 * N + 1]), "min")[0])
            P_.hist.append(c)
            Rt = P_.R_tilde
            beta = float(self.betas[t])
            o = dict(t=t, beta=beta, R_tilde=Rt, sum_E=int(sums[0]), sum_E2=int(sums[1]), E_min=Emin)
            o["mean_E"] = float(sums[0]) / float(Rt)
            o["var_E"] = float(sums[1]) / float(Rt) - o["mean_E"] * o["mean_E"]
            o["minus_beta_F"] = float(N) * math.log(2.0) + P_.lnQ_sum
            if t == 0 or Emin < P_.E0:
                P_.E0 = Emin
            o["E0"] = P_.E0
            o["g0_tilde"] = float(c[(P_.E0 + 3 * N) // 2]) / float(Rt)
            o["g0_bar"] = 2.0 * math.exp(-(beta * float(P_.E0)) - o["minus_beta_F"])
            sum_eta2, n_fam, m = self._families(P_)
            S_f = 0.0
            for eta in range(1, m.size):     # ascending family size, as the single-process oracle sums
                if m[eta] == 0:
                    continue
                nu = eta / Rt
                S_f = S_f - float(m[eta]) * (nu * math.log(nu))
            o.update(sum_eta2=sum_eta2, n_families=n_fam, S_f=S_f, rho_t=float(sum_eta2) / float(Rt),
                     rho_s=float(Rt) / math.exp(S_f), q_pairs=0, q_abs_le_02=0, I02=0.0)
            if t > 0:
                o.update(P_._step_fields)
            o["family_sizes"] = m
            if t == 0:
                P_.obs.append(o)
            else:
                P_.obs[t] = o
        if self.n_pop == 2:
            A, B = self.pops
            pairs = min(A.R_tilde, B.R_tilde)
            n_loc = max(0, min(A.s.shape[0], B.s.shape[0], pairs - A.lo))
            Q = (A.s[:n_loc].astype(np.int64) * B.s[:n_loc].astype(np.int64)).sum(axis=1)
            nb = self.q_bins
            bins = ((Q + N) * (nb - 1) + N) // (2 * N)
            qh = self._allreduce(np.bincount(bins, minlength=nb)[:nb])
            small = int(self._allreduce(np.array([(5 * np.abs(Q) <= N).sum()]))[0])
            self.qhist.append(qh)
            for P_ in self.pops:
                P_.obs[t].update(q_pairs=pairs, q_abs_le_02=small, I02=float(small) / float(pairs) if pairs else 0.0)

    # ------------------------------------------------------------ inspection
    def gather_population(self, p: int = 0):
        """(spins [R~, N], labels, energies) of population p in slot order, on every rank."""
        import torch.distributed as dist
        parts = [None] * self.P
        P_ = self.pops[p]
        dist.all_gather_object(parts, (P_.lo, P_.s, P_.lab, P_.E))
        parts.sort(key=lambda x: x[0])
        return (np.concatenate([x[1] for x in parts]), np.concatenate([x[2] for x in parts]),
                np.concatenate([x[3] for x in parts]))

    def gather_counts(self, p: int = 0) -> np.ndarray:
        """Copy numbers of the last resampling, in old-slot order, on every rank."""
        import torch.distributed as dist
        parts = [None] * self.P
        dist.all_gather_object(parts, self.pops[p].counts)
        return np.concatenate(parts)
