"""Writes the oracle-generated fixtures of this directory (calls only ``oracle``).

    python tests/golden/make_golden.py

philox_kat.txt        Philox4x32-10 blocks for fixed counters and keys (the oracle's
                      generator, itself pinned against an independent implementation).
c1_trajectory.txt     per-step integer observables of the L=4, R=1000, 51-temperature
                      +-1 workload (couplings seed 1, run seed 1001, 10 sweeps).
gauss_trajectory.txt  the same for a small Gaussian-coupling run with two populations
                      (L=6, R=800, 9 temperatures to beta=3, 3 sweeps, seeds 3 and 4).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.abspath(os.path.join(HERE, "..", "..")))

import oracle  # noqa: E402

PM1_FIELDS = ("t", "R_tilde", "sum_E", "sum_E2", "E_min", "culled", "sum_eta2", "n_families", "E0")
GAUSS_FIELDS = ("t", "R_tilde", "sum_E", "E_min", "culled", "sum_eta2", "n_families", "E0", "q_pairs", "ql_sum")


def philox_kat():
    rows = []
    for i in range(32):
        ctr = [(i * 2654435761) & 0xFFFFFFFF, i, (i * i * 40503) & 0xFFFFFFFF, (0xFFFFFFFF - i) & 0xFFFFFFFF]
        key = [(i * 0x9E3779B9) & 0xFFFFFFFF, (i * 0xBB67AE85 + 7) & 0xFFFFFFFF]
        out = oracle.philox(ctr, key)
        rows.append(" ".join(f"{v:08x}" for v in ctr + key + [int(x) for x in out]))
    return "# ctr0 ctr1 ctr2 ctr3 key0 key1 -> out0 out1 out2 out3 (hex)\n" + "\n".join(rows) + "\n"


def c1_trajectory():
    betas = np.array([t * 5.0 / 50 for t in range(51)])
    run = oracle.Run(oracle.RunConfig(L=4, R=1000, disorder_seed=1, run_seed=1001, betas=betas, n_sweeps=10))
    run.run()
    lines = ["# " + " ".join(PM1_FIELDS)]
    for t in range(51):
        o = run.obs(t)
        lines.append(" ".join(str(int(o[k])) for k in PM1_FIELDS))
    return "\n".join(lines) + "\n"


def gauss_trajectory():
    betas = np.linspace(0.0, 3.0, 9)
    run = oracle.GRun(oracle.RunConfig(L=6, R=800, disorder_seed=3, run_seed=4, betas=betas, n_sweeps=3, n_pop=2))
    run.run()
    lines = ["# " + " ".join(GAUSS_FIELDS)]
    for t in range(9):
        o = run.obs(t, 0)
        lines.append(" ".join(str(int(o[k])) for k in GAUSS_FIELDS))
    return "\n".join(lines) + "\n"


FILES = {"philox_kat.txt": philox_kat, "c1_trajectory.txt": c1_trajectory, "gauss_trajectory.txt": gauss_trajectory}

if __name__ == "__main__":
    oracle.build()
    for name, fn in FILES.items():
        with open(os.path.join(HERE, name), "w") as f:
            f.write(fn())
        print("wrote", name)
