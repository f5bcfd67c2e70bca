"""The GPU path against stored oracle trajectories (tests/golden, written by
make_golden.py from the oracle alone): no oracle runs at test time."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def pa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_02146_gb300 import build, pa as pa_mod
    build.build()
    return pa_mod


def table(name):
    lines = open(os.path.join(HERE, name)).read().splitlines()
    return lines[0].lstrip("# ").split(), [list(map(int, line.split())) for line in lines[1:]]


def test_c1_trajectory(pa):
    from paper_1711_02146_gb300.workloads import C1
    fields, rows = table("c1_trajectory.txt")
    run = pa.Run.from_workload(C1)
    run.run()
    for row in rows:
        o = run.obs(row[0])
        assert [int(o[k]) for k in fields] == row, f"t={row[0]}"


def test_gaussian_trajectory(pa):
    fields, rows = table("gauss_trajectory.txt")
    run = pa.Run(6, 800, 3, 4, np.linspace(0.0, 3.0, 9), n_sweeps=3, n_pop=2, model=pa.PA_MODEL_GAUSS)
    run.run()
    for row in rows:
        o = run.gobs(row[0], 0)
        assert [int(o[k]) for k in fields] == row, f"t={row[0]}"
