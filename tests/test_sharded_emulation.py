"""The sharded step (a population split across ranks, gloo on CPU) reproduces the
single-process oracle bit for bit: spins, labels, energies, copy numbers, level
and overlap histograms, family statistics and every observable, at 2 and 3
ranks, with families that straddle rank boundaries."""
import os
import socket
import traceback

import numpy as np
import pytest

CASES = {
    # P ranks, L, R, temperatures, beta_max, sweeps, populations
    "two_ranks_one_population": (2, 4, 200, 6, 2.0, 2, 1),
    "three_ranks_two_populations": (3, 4, 150, 5, 3.0, 1, 2),
    "three_ranks_strong_culling": (3, 2, 90, 4, 4.0, 1, 1),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _compare(sh, ref, t):
    """Mismatches between the sharded run (gathered) and the oracle at step t."""
    bad = []
    for p in range(sh.n_pop):
        s, lab, E = sh.gather_population(p)
        rs, rlab, rE = ref.population(p)
        if s.shape != rs.shape or not np.array_equal(s, rs):
            bad.append(f"t={t} pop {p}: spins")
        if not np.array_equal(lab, rlab):
            bad.append(f"t={t} pop {p}: labels")
        if not np.array_equal(E, rE):
            bad.append(f"t={t} pop {p}: energies")
        if t > 0 and not np.array_equal(sh.gather_counts(p), ref.last_counts(p)):
            bad.append(f"t={t} pop {p}: copy numbers")
        if not np.array_equal(sh.pops[p].hist[t], ref.energy_hist(t, p)):
            bad.append(f"t={t} pop {p}: level histogram")
        o, r = sh.pops[p].obs[t], ref.obs(t, p)
        for k, v in o.items():
            if k != "family_sizes" and k in r and r[k] != v:
                bad.append(f"t={t} pop {p}: {k} {v!r} vs {r[k]!r}")
        eta, m = ref.family_hist(p)
        mine = o["family_sizes"]
        nz = np.nonzero(mine)[0]
        if not (np.array_equal(nz, eta) and np.array_equal(mine[nz], m)):
            bad.append(f"t={t} pop {p}: family-size histogram")
    if sh.n_pop == 2 and not np.array_equal(sh.qhist[t], ref.q_hist(t)):
        bad.append(f"t={t}: overlap histogram")
    return bad


def _rank(rank, case, port, out):
    try:
        import torch.distributed as dist
        P, L, R, T, bmax, S, n_pop = CASES[case]
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=rank, world_size=P)
        import oracle
        from oracle.sharded import ShardedRun
        betas = np.array([t * bmax / (T - 1) for t in range(T)])
        sh = ShardedRun(L, R, disorder_seed=5, run_seed=77, betas=betas, n_sweeps=S, n_pop=n_pop)
        ref = oracle.Run(oracle.RunConfig(L=L, R=R, disorder_seed=5, run_seed=77, betas=betas, n_sweeps=S,
                                          n_pop=n_pop))
        bad = _compare(sh, ref, 0)
        straddle = 0
        for t in range(1, T):
            sh.step()
            ref.step()
            bad += _compare(sh, ref, t)
            # families that span a rank boundary: the first label of a rank equals the last of the one before
            for P_ in sh.pops:
                edge = sh._allgather(np.array([P_.lab[0] if P_.lab.size else -1,
                                               P_.lab[-1] if P_.lab.size else -2]))
                straddle += int(sum(edge[q, 0] == edge[q - 1, 1] for q in range(1, P)))
        dist.barrier()
        out.put((rank, bad, straddle))
        dist.destroy_process_group()
    except Exception:
        out.put((rank, [traceback.format_exc()], 0))


@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_run_matches_single_process(oracle_lib, case):
    import torch.multiprocessing as mp
    P = CASES[case][0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, case, port, q)) for r in range(P)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
    for rank, bad, _ in res:
        assert not bad, f"rank {rank}: " + "; ".join(bad[:8])
    assert all(p.exitcode == 0 for p in procs)
    assert res[0][2] > 0, "no family crossed a rank boundary: the boundary join was not exercised"
