"""A population split across ranks on the GPU (pa_shard, §I: PA on computing
clusters): 2 and 3 processes, each holding a block of every population in its
own CUDA context, the host exchanges over gloo.  Every random word is addressed by
global slot, so the gathered populations, the copy numbers of the last step, the
overlap histograms and every observable must be those of one process
(pa_create / pa_step on the whole population) bit for bit.  The ranks share one
GPU here, their kernels never wait on each other (the exchanges are on the host),
and no multi-GPU run has been measured."""
import os
import pickle
import socket
import traceback

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = {
    # ranks, L, R, temperatures, beta_max, sweeps, populations, disorder seed
    "two_ranks_two_populations": (2, 8, 5000, 6, 2.5, 2, 2, 4),
    "three_ranks_strong_culling": (3, 4, 3500, 5, 6.0, 1, 1, 7),
    "three_ranks_L6": (3, 6, 4100, 7, 3.0, 3, 1, 9),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _betas(T, bmax):
    return np.array([t * bmax / (T - 1) for t in range(T)])


def _rank(rank, case, port, out_dir):
    import datetime

    import torch.distributed as dist
    P, L, R, T, bmax, S, n_pop, seed = CASES[case]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=P, timeout=datetime.timedelta(seconds=120))
    res = {"error": None}
    try:
        from paper_1711_02146_gb300 import pa
        sh = pa.Shard(L, R, seed, 100 + seed, _betas(T, bmax), n_sweeps=S, n_pop=n_pop)
        obs = [[sh.obs(0, p) for p in range(n_pop)]]
        q = [sh.q_hist(0)] if n_pop == 2 else []
        extents = []
        while True:
            lo_old = [sh.extent(p)[0] for p in range(n_pop)]
            if sh.step() != 0:
                break
            obs.append([sh.obs(sh.t, p) for p in range(n_pop)])
            if n_pop == 2:
                q.append(sh.q_hist(sh.t))
            extents.append(lo_old)
        res["obs"], res["q"] = obs, q
        res["lo"] = [sh.extent(p)[0] for p in range(n_pop)]
        res["pop"] = [sh.local.population(p) for p in range(n_pop)]
        res["counts"] = [sh.local.copy_counts(p) for p in range(n_pop)]
        sh.close()
    except Exception:
        res["error"] = traceback.format_exc()
    with open(os.path.join(out_dir, f"rank{rank}.pkl"), "wb") as f:
        pickle.dump(res, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_run_is_the_one_process_run(case, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    from paper_1711_02146_gb300 import build, pa
    build.build()
    P, L, R, T, bmax, S, n_pop, seed = CASES[case]
    mp.start_processes(_rank, args=(case, _free_port(), str(tmp_path)), nprocs=P, join=True, start_method="spawn")
    parts = []
    for r in range(P):
        with open(tmp_path / f"rank{r}.pkl", "rb") as f:
            res = pickle.load(f)
        assert res["error"] is None, f"rank {r}:\n{res['error']}"
        parts.append(res)
    ref = pa.Run(L, R, seed, 100 + seed, _betas(T, bmax), n_sweeps=S, n_pop=n_pop)
    ref.run()
    for t in range(T):
        for p in range(n_pop):
            want = ref.obs(t, p)
            for r in range(P):
                assert parts[r]["obs"][t][p] == want, f"rank {r} t={t} pop {p}"
        if n_pop == 2:
            for r in range(P):
                assert np.array_equal(parts[r]["q"][t], ref.q_hist(t)), f"overlap histogram t={t}"
    for p in range(n_pop):
        order = sorted(range(P), key=lambda r: parts[r]["lo"][p])
        spins = np.concatenate([parts[r]["pop"][p][0] for r in order])
        labels = np.concatenate([parts[r]["pop"][p][1] for r in order])
        energies = np.concatenate([parts[r]["pop"][p][2] for r in order])
        rs, rlab, rE = ref.population(p)
        assert spins.shape == rs.shape and np.array_equal(spins, rs), f"pop {p}: spins"
        assert np.array_equal(labels, rlab) and np.array_equal(energies, rE), f"pop {p}: labels, energies"
        # the copy numbers of the last resampling, old slots of every rank in rank order
        counts = np.concatenate([parts[r]["counts"][p] for r in range(P)])
        assert np.array_equal(counts, ref.copy_counts(p)), f"pop {p}: copy numbers"
    ref.close()
