"""GB300-native population annealing (Amey & Machta, arXiv:1711.02146).

The hot path — Metropolis sweeps, reweighting, nearest-integer resampling and the
estimator reductions — runs in hand-written sm_103a CUDA kernels inside
``libpa.so``; ``pa`` is its thin ctypes binding, ``drivers`` the paper's host
procedures built on runs, ``workloads`` seeded input recipes.

Typical use::

    from paper_1711_02146_gb300 import build, pa
    from paper_1711_02146_gb300.workloads import Workload, linear_betas
    build.build()                                   # compiles libpa.so in place (sm_103a)
    run = pa.Run(L=10, R=100_000, disorder_seed=3, run_seed=1,
                 betas=linear_betas(101, 5.0), n_sweeps=10)
    run.run()                                       # all temperature steps on the GPU
    o = run.obs(run.t)                              # -beta F, <E>, rho_t, S_f, g0, ...
    # adaptive schedule at constant culling fraction (§IV.B):
    run = pa.Run(10, 1_000_000, 3, 1, None, n_temps=4096, beta_max=5.0, eps_target=0.272)
    # Gaussian couplings (the paper's model), two populations for q and q_l:
    run = pa.Run(8, 50_000, 7, 1, linear_betas(51, 3.0), n_pop=2, model=pa.PA_MODEL_GAUSS)
    run.run(); g = run.gobs(run.t)                  # ..., ql_mean, e_l, delta_KY
    # many runs at once: pa.Batch([...workloads]).run(), or pa.Server(budget) for a stream
"""
