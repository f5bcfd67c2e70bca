"""GB300-native population annealing (Amey & Machta, arXiv:1711.02146).

The hot path — Metropolis sweeps, reweighting, nearest-integer resampling and the
estimator reductions — runs in hand-written sm_103a CUDA kernels inside
``libpa.so``; ``pa`` is its thin ctypes binding.
"""
