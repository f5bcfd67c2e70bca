"""Thin ctypes binding of libpa.so (the C ABI declared in include/pa.h).

Argument marshalling only: every step of a run executes in the library's CUDA
kernels.  There is no CPU fallback — importing this module without a built
libpa.so, or creating a run without a CUDA device, raises.

PyTorch is optional here: a torch CUDA stream may be passed as ``stream``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpa.so")

# Runs on separate streams (Batch, Server) overlap on the device only as far as its
# hardware work queues allow; CUDA reads the queue count when it creates the
# context, so this default (the driver's own is 8) applies only when this module is
# imported before the process's first CUDA call, and never overrides a user's value.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

PA_OK, PA_DONE = 0, 1
PA_ERR_INVALID, PA_ERR_NOMEM, PA_ERR_CAPACITY, PA_ERR_TIMEOUT = -1, -2, -3, -4
PA_ERR_CUDA, PA_ERR_STATE, PA_ERR_EXTINCT = -5, -6, -7


class PAError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {status} ({strerror(status)})")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32),
        ("n_pop", ctypes.c_int32),
        ("R", ctypes.c_int64),
        ("R_cap", ctypes.c_int64),
        ("disorder_seed", ctypes.c_uint64),
        ("run_seed", ctypes.c_uint64),
        ("n_temps", ctypes.c_int32),
        ("betas", ctypes.POINTER(ctypes.c_double)),
        ("beta_max", ctypes.c_double),
        ("eps_target", ctypes.c_double),
        ("n_sweeps", ctypes.c_int32),
        ("sweeps_per_step", ctypes.POINTER(ctypes.c_int32)),
        ("q_bins", ctypes.c_int32),
        ("model", ctypes.c_int32),
    ]


PA_MODEL_PM1, PA_MODEL_GAUSS = 0, 1
PA_BATCH_FUSED, PA_BATCH_STREAMS = 0, 1


class GObs(ctypes.Structure):
    """Observables of a Gaussian-coupling run (pa_gobs)."""
    _fields_ = [
        ("t", ctypes.c_int32), ("beta", ctypes.c_double), ("dbeta", ctypes.c_double),
        ("R_tilde", ctypes.c_int64), ("sum_E", ctypes.c_int64), ("sum_E2", ctypes.c_double),
        ("E_min", ctypes.c_int64), ("mean_E", ctypes.c_double), ("var_E", ctypes.c_double),
        ("E_min_prev", ctypes.c_int64), ("S_prime", ctypes.c_double), ("lnQ", ctypes.c_double),
        ("minus_beta_F", ctypes.c_double), ("eps_expected", ctypes.c_double), ("culled", ctypes.c_int64),
        ("sum_eta2", ctypes.c_int64), ("n_families", ctypes.c_int64), ("rho_t", ctypes.c_double),
        ("S_f", ctypes.c_double), ("rho_s", ctypes.c_double), ("E0", ctypes.c_int64),
        ("g0_tilde", ctypes.c_double), ("g0_bar", ctypes.c_double), ("q_pairs", ctypes.c_int64),
        ("q_abs_le_02", ctypes.c_int64), ("I02", ctypes.c_double), ("ql_sum", ctypes.c_int64),
        ("ql_mean", ctypes.c_double), ("e_l", ctypes.c_double), ("delta_KY", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Obs(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_int32),
        ("beta", ctypes.c_double),
        ("dbeta", ctypes.c_double),
        ("R_tilde", ctypes.c_int64),
        ("sum_E", ctypes.c_int64),
        ("sum_E2", ctypes.c_int64),
        ("E_min", ctypes.c_int32),
        ("mean_E", ctypes.c_double),
        ("var_E", ctypes.c_double),
        ("kmin_prev", ctypes.c_int32),
        ("S_prime", ctypes.c_double),
        ("lnQ", ctypes.c_double),
        ("minus_beta_F", ctypes.c_double),
        ("eps_expected", ctypes.c_double),
        ("culled", ctypes.c_int64),
        ("sum_eta2", ctypes.c_int64),
        ("n_families", ctypes.c_int64),
        ("rho_t", ctypes.c_double),
        ("S_f", ctypes.c_double),
        ("rho_s", ctypes.c_double),
        ("E0", ctypes.c_int32),
        ("g0_tilde", ctypes.c_double),
        ("g0_bar", ctypes.c_double),
        ("q_pairs", ctypes.c_int64),
        ("q_abs_le_02", ctypes.c_int64),
        ("I02", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


PHASES = ("reweight", "resample", "sweep", "family", "overlap")


class Stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("h2d_bytes", ctypes.c_int64),
        ("d2h_bytes", ctypes.c_int64),
        ("updates", ctypes.c_int64),
        ("phase_ms", ctypes.c_double * 5),
        ("phase_count", ctypes.c_int64 * 5),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k in ("steps", "kernel_launches", "h2d_bytes", "d2h_bytes", "updates")}
        d["phase_ms"] = dict(zip(PHASES, list(self.phase_ms)))
        d["phase_count"] = dict(zip(PHASES, list(self.phase_count)))
        return d


class SweepShape(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("words", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("smem_bytes", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None

# Every entry point declared in include/pa.h, with its ctypes signature.
_i8p = ctypes.POINTER(ctypes.c_int8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p
_ALLREDUCE = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64)
_ALLGATHER = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                              ctypes.POINTER(ctypes.c_int64))
_XFER = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64)


class Comm(ctypes.Structure):
    """pa_comm: the host exchanges of a sharded run."""
    _fields_ = [("user", ctypes.c_void_p), ("allreduce_i64", _ALLREDUCE), ("allgather_i64", _ALLGATHER),
                ("send", _XFER), ("recv", _XFER)]


SIGNATURES = {
    "pa_create": (ctypes.c_int, [ctypes.POINTER(Config), _vp, ctypes.POINTER(_vp)]),
    "pa_step": (ctypes.c_int, [_vp]),
    "pa_run": (ctypes.c_int, [_vp]),
    "pa_current_step": (ctypes.c_int32, [_vp]),
    "pa_observables": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Obs)]),
    "pa_energy_hist": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _i64p, ctypes.c_int64]),
    "pa_q_hist": (ctypes.c_int, [_vp, ctypes.c_int32, _i64p, ctypes.c_int64]),
    "pa_family_hist": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int64, _i64p, _i64p, _i64p]),
    "pa_population_size": (ctypes.c_int, [_vp, ctypes.c_int32, _i64p]),
    "pa_get_replicas": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _i8p, _i32p, _i32p]),
    "pa_get_copy_counts": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, ctypes.c_int64, _i64p]),
    "pa_get_parents": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, ctypes.c_int64, _i64p]),
    "pa_get_couplings": (ctypes.c_int, [_vp, _i8p, ctypes.c_int64]),
    "pa_beta": (ctypes.c_double, [_vp, ctypes.c_int32]),
    "pa_stats_reset": (ctypes.c_int, [_vp, ctypes.c_int]),
    "pa_debug_lookback": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "pa_debug_bisect": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "pa_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
    "pa_sync": (ctypes.c_int, [_vp]),
    "pa_destroy": (ctypes.c_int, [_vp]),
    "pa_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pa_footprint": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_size_t)]),
    "pa_batch_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int32, ctypes.POINTER(_vp)]),
    "pa_batch_run": (ctypes.c_int, [_vp]),
    "pa_batch_ctx": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(_vp)]),
    "pa_batch_destroy": (ctypes.c_int, [_vp]),
    "pa_batch_set_mode": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "pa_batch_launches": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "pa_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_vp)]),
    "pa_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_uint64)]),
    "pa_server_poll": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "pa_server_result": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(Obs),
                                        ctypes.POINTER(ctypes.c_int32)]),
    "pa_server_gresult": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(GObs),
                                         ctypes.POINTER(ctypes.c_int32)]),
    "pa_server_load": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "pa_server_destroy": (ctypes.c_int, [_vp]),
    "pa_gobservables": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(GObs)]),
    "pa_get_genergies": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _i64p]),
    "pa_ql_hist": (ctypes.c_int, [_vp, ctypes.c_int32, _i64p, ctypes.c_int64]),
    "pa_get_gcouplings": (ctypes.c_int, [_vp, _i32p, ctypes.c_int64]),
    "pa_checkpoint": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "pa_restore": (ctypes.c_int, [ctypes.POINTER(Config), _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    "pa_sweep_shapes": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(SweepShape), ctypes.c_int32, _i32p]),
    "pa_sweep_select": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
    "pa_sweep_selected": (ctypes.c_int, [ctypes.c_int32, _i32p]),
    "pa_sweep_plan": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "pa_sweep_autotune": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_int32, _i32p]),
    "pa_resample_counts_noalloc": (ctypes.c_int, [_vp, ctypes.c_int64, _vp, _vp, ctypes.c_int32, ctypes.c_uint64,
                                                   ctypes.c_int32, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp,
                                                   _vp]),
    "pa_shard_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Comm),
                                       _vp, ctypes.POINTER(_vp)]),
    "pa_shard_step": (ctypes.c_int, [_vp]),
    "pa_shard_observables": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Obs)]),
    "pa_shard_local": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "pa_shard_extent": (ctypes.c_int, [_vp, ctypes.c_int32, _i64p, _i64p]),
    "pa_shard_q_hist": (ctypes.c_int, [_vp, ctypes.c_int32, _i64p, ctypes.c_int64]),
    "pa_shard_destroy": (ctypes.c_int, [_vp]),
    "pa_bench_int_throughput": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
}

NOALLOC_MAX_SLOTS = 4096 * 1024


def sweep_shapes(L: int) -> list:
    """Launch shapes compiled for the sweep kernel at size L, default first (no GPU needed)."""
    n = ctypes.c_int32()
    _check("pa_sweep_shapes", lib().pa_sweep_shapes(L, None, 0, ctypes.byref(n)))
    arr = (SweepShape * n.value)()
    _check("pa_sweep_shapes", lib().pa_sweep_shapes(L, arr, n.value, ctypes.byref(n)))
    return [a.as_dict() for a in arr]


def sweep_select(L: int, index: int) -> None:
    """Shape `index` of L for runs created afterwards on the current device (-1: default)."""
    _check("pa_sweep_select", lib().pa_sweep_select(L, index))


def sweep_selected(L: int) -> int:
    i = ctypes.c_int32()
    _check("pa_sweep_selected", lib().pa_sweep_selected(L, ctypes.byref(i)))
    return i.value


def sweep_autotune(L: int, R: int, launches: int = 5):
    """Times every sweep shape of L on a scratch run of R replicas and selects the
    fastest on the current device; returns (index, [ms per launch of each shape])."""
    n = len(sweep_shapes(L))
    ms = (ctypes.c_double * n)()
    best = ctypes.c_int32()
    _check("pa_sweep_autotune", lib().pa_sweep_autotune(L, R, launches, ms, n, ctypes.byref(best)))
    return best.value, list(ms)


def resample_counts_noalloc(levels, n_old, fl, thr, n_levels, run_seed, pop, t, counts, parents, parents_cap, n_new,
                            stream=None) -> int:
    """pa_resample_counts_noalloc on caller-owned device buffers (device pointers as ints,
    e.g. torch tensors' data_ptr()); returns the status code."""
    return int(lib().pa_resample_counts_noalloc(levels, n_old, fl, thr, n_levels, run_seed, pop, t, counts, parents,
                                                parents_cap, n_new, _stream_handle(stream)))


PROBES = {"lop3": 0, "iadd": 1, "imad": 2, "mulwide": 3, "philox": 4, "mulwide_add": 5, "lop3_iadd": 6,
          "philox_lop3": 7}


def int_throughput(kind: str, iters: int = 4096, blocks: int = 0, threads: int = 256):
    """Integer-throughput probe (include/pa_bench.h): returns operations per second
    (Philox words per second for kind="philox")."""
    if blocks <= 0:
        import torch
        blocks = 16 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    ms, ops = ctypes.c_double(), ctypes.c_double()
    _check("pa_bench_int_throughput", lib().pa_bench_int_throughput(PROBES[kind], iters, blocks, threads,
                                                                    ctypes.byref(ms), ctypes.byref(ops)))
    return ops.value / (ms.value / 1e3)


def lib():
    """Loads libpa.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1711_02146_gb300.build` "
                              "(or __graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    try:
        return lib().pa_strerror(status).decode()
    except ImportError:
        return "?"


def _check(fn: str, rc: int) -> int:
    if rc < 0:
        raise PAError(fn, rc)
    return rc


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class _ConfigHolder:
    """A pa_config plus the arrays it points to (kept alive with it)."""

    def __init__(self, L, R, disorder_seed, run_seed, betas=None, n_temps=0, beta_max=0.0, eps_target=0.0,
                 n_sweeps=10, sweeps_per_step=None, n_pop=1, q_bins=65, R_cap=0, model=0):
        self.betas = None if betas is None else np.ascontiguousarray(betas, dtype=np.float64)
        self.sweeps = None if sweeps_per_step is None else np.ascontiguousarray(sweeps_per_step, dtype=np.int32)
        c = Config()
        c.L, c.n_pop, c.R, c.R_cap = L, n_pop, R, R_cap
        c.disorder_seed, c.run_seed = disorder_seed, run_seed
        c.n_temps = len(self.betas) if self.betas is not None else n_temps
        c.betas = _p(self.betas, ctypes.c_double) if self.betas is not None else None
        c.beta_max, c.eps_target, c.n_sweeps = beta_max, eps_target, n_sweeps
        c.sweeps_per_step = _p(self.sweeps, ctypes.c_int32) if self.sweeps is not None else None
        c.q_bins = q_bins
        c.model = model
        self.cfg = c

    @classmethod
    def from_workload(cls, w):
        return cls(w.L, w.R, w.disorder_seed, w.run_seed, w.betas, n_temps=w.n_temps, beta_max=w.beta_max,
                   eps_target=w.eps_target, n_sweeps=w.n_sweeps, sweeps_per_step=w.sweeps_per_step, n_pop=w.n_pop,
                   q_bins=w.q_bins, R_cap=w.R_cap, model=w.model)


def footprint(w) -> int:
    """Device bytes a run of workload w allocates (pa_footprint)."""
    h = _ConfigHolder.from_workload(w)
    b = ctypes.c_size_t()
    _check("pa_footprint", lib().pa_footprint(ctypes.byref(h.cfg), ctypes.byref(b)))
    return b.value


class _View:
    """Observables of a borrowed pa_ctx (a run inside a batch)."""

    def __init__(self, handle, owner, L, n_pop, q_bins):
        self._h, self._owner = handle, owner
        self.L, self.N, self.n_pop, self.q_bins = L, L ** 3, n_pop, q_bins
        self.n_levels = 3 * self.N + 1


class Batch:
    """Many independent runs advanced together (pa_batch): by default in rounds of one
    CUDA graph launch for all runs that qualify (``mode="fused"``), or each run on its
    own stream (``mode="streams"``)."""

    MODES = {"fused": PA_BATCH_FUSED, "streams": PA_BATCH_STREAMS}

    def __init__(self, workloads, mode: str = "fused"):
        self.workloads = list(workloads)
        self._holders = [_ConfigHolder.from_workload(w) for w in self.workloads]
        arr = (Config * len(self._holders))(*[h.cfg for h in self._holders])
        self._arr = arr
        h = _vp()
        _check("pa_batch_create", lib().pa_batch_create(arr, len(self._holders), ctypes.byref(h)))
        self._h = h
        _check("pa_batch_set_mode", lib().pa_batch_set_mode(self._h, self.MODES[mode]))

    def run(self) -> None:
        _check("pa_batch_run", lib().pa_batch_run(self._h))

    def launches(self) -> dict:
        """Kernels and CUDA graphs launched by run() so far."""
        k, g = ctypes.c_int64(), ctypes.c_int64()
        _check("pa_batch_launches", lib().pa_batch_launches(self._h, ctypes.byref(k), ctypes.byref(g)))
        return {"kernels": k.value, "graphs": g.value}

    def run_view(self, i: int) -> "Run":
        v = _vp()
        _check("pa_batch_ctx", lib().pa_batch_ctx(self._h, i, ctypes.byref(v)))
        w = self.workloads[i]
        return Run._borrowed(v, self, w.L, w.n_pop, w.q_bins, w.model)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().pa_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (pa_server): FIFO admission by device-memory footprint."""

    def __init__(self, mem_budget: int, max_active: int = 256, steps_per_poll: int = 1):
        h = _vp()
        _check("pa_server_create", lib().pa_server_create(mem_budget, max_active, steps_per_poll, ctypes.byref(h)))
        self._h = h
        self._done = (ctypes.c_uint64 * 4096)()

    def submit(self, w) -> int:
        holder = _ConfigHolder.from_workload(w)
        rid = ctypes.c_uint64()
        _check("pa_server_submit", lib().pa_server_submit(self._h, ctypes.byref(holder.cfg), ctypes.byref(rid)))
        return rid.value

    def poll(self):
        n = ctypes.c_int32()
        _check("pa_server_poll", lib().pa_server_poll(self._h, self._done, len(self._done), ctypes.byref(n)))
        return [int(self._done[i]) for i in range(n.value)]

    def result(self, rid: int, pop: int = 0):
        """(observables dict, last step) of a finished request; raises PAError with the
        request's own status if it failed."""
        o = Obs()
        t = ctypes.c_int32()
        _check("pa_server_result", lib().pa_server_result(self._h, rid, pop, ctypes.byref(o), ctypes.byref(t)))
        return o.as_dict(), t.value

    def gresult(self, rid: int, pop: int = 0):
        """(Gaussian observables dict, last step) of a finished Gaussian-coupling request."""
        o = GObs()
        t = ctypes.c_int32()
        _check("pa_server_gresult", lib().pa_server_gresult(self._h, rid, pop, ctypes.byref(o), ctypes.byref(t)))
        return o.as_dict(), t.value

    def load(self):
        q, a = ctypes.c_int32(), ctypes.c_int32()
        _check("pa_server_load", lib().pa_server_load(self._h, ctypes.byref(q), ctypes.byref(a)))
        return q.value, a.value

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().pa_server_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Run:
    """One population annealing run on the GPU (a ``pa_ctx``)."""

    @classmethod
    def _borrowed(cls, handle, owner, L, n_pop, q_bins, model=0):
        r = cls.__new__(cls)
        r._h, r._owner, r._borrowed_view = handle, owner, True
        r.L, r.N, r.n_pop, r.q_bins = L, L ** 3, n_pop, q_bins
        r.n_levels = 3 * r.N + 1
        r.n_temps = None
        r.model = model
        return r

    def __init__(self, L: int, R: int, disorder_seed: int, run_seed: int, betas=None, *, n_temps: int = 0,
                 beta_max: float = 0.0, eps_target: float = 0.0, n_sweeps: int = 10, sweeps_per_step=None,
                 n_pop: int = 1, q_bins: int = 65, R_cap: int = 0, stream=None, checkpoint: bytes = None,
                 model: int = 0):
        """Creates a run (pa_create), or, given `checkpoint` (bytes from Run.checkpoint of a
        run with this configuration), restores it (pa_restore)."""
        self.L, self.N, self.n_pop, self.q_bins = L, L ** 3, n_pop, q_bins
        self.n_levels = 3 * self.N + 1
        self._betas = None if betas is None else np.ascontiguousarray(betas, dtype=np.float64)
        self._sweeps = None if sweeps_per_step is None else np.ascontiguousarray(sweeps_per_step, dtype=np.int32)
        c = Config()
        c.L, c.n_pop, c.R, c.R_cap = L, n_pop, R, R_cap
        c.disorder_seed, c.run_seed = disorder_seed, run_seed
        c.n_temps = len(self._betas) if self._betas is not None else n_temps
        c.betas = _p(self._betas, ctypes.c_double) if self._betas is not None else None
        c.beta_max, c.eps_target, c.n_sweeps = beta_max, eps_target, n_sweeps
        c.sweeps_per_step = _p(self._sweeps, ctypes.c_int32) if self._sweeps is not None else None
        c.q_bins = q_bins
        c.model = model
        self.model = model
        self.n_temps = c.n_temps
        h = _vp()
        if checkpoint is None:
            _check("pa_create", lib().pa_create(ctypes.byref(c), _stream_handle(stream), ctypes.byref(h)))
        else:
            buf = ctypes.create_string_buffer(bytes(checkpoint), len(checkpoint))
            _check("pa_restore", lib().pa_restore(ctypes.byref(c), buf, len(checkpoint), _stream_handle(stream),
                                                  ctypes.byref(h)))
        self._h = h

    def checkpoint(self) -> bytes:
        """The run's state after its last step (pa_checkpoint)."""
        n = ctypes.c_size_t()
        rc = lib().pa_checkpoint(self._h, None, 0, ctypes.byref(n))
        if rc != PA_ERR_CAPACITY:
            _check("pa_checkpoint", rc)
        buf = ctypes.create_string_buffer(n.value)
        _check("pa_checkpoint", lib().pa_checkpoint(self._h, buf, n.value, ctypes.byref(n)))
        return buf.raw[: n.value]

    @classmethod
    def from_workload(cls, w, stream=None, **over):
        kw = dict(n_temps=w.n_temps, beta_max=w.beta_max, eps_target=w.eps_target, n_sweeps=w.n_sweeps,
                  sweeps_per_step=w.sweeps_per_step, n_pop=w.n_pop, q_bins=w.q_bins, R_cap=w.R_cap, model=w.model)
        kw.update(over)
        return cls(w.L, w.R, w.disorder_seed, w.run_seed, w.betas, stream=stream, **kw)

    def close(self):
        if getattr(self, "_borrowed_view", False):
            return
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().pa_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- stepping
    def step(self) -> int:
        return _check("pa_step", lib().pa_step(self._h))

    def run(self) -> None:
        _check("pa_run", lib().pa_run(self._h))

    def sync(self) -> None:
        _check("pa_sync", lib().pa_sync(self._h))

    @property
    def t(self) -> int:
        return int(lib().pa_current_step(self._h))

    def beta(self, t: int) -> float:
        return float(lib().pa_beta(self._h, t))

    def stats_reset(self, timing: bool = False) -> None:
        _check("pa_stats_reset", lib().pa_stats_reset(self._h, 1 if timing else 0))

    def stats(self) -> dict:
        st = Stats()
        _check("pa_get_stats", lib().pa_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    # ---- results
    def obs(self, t: int, pop: int = 0) -> dict:
        o = Obs()
        _check("pa_observables", lib().pa_observables(self._h, t, pop, ctypes.byref(o)))
        return o.as_dict()

    def energy_hist(self, t: int, pop: int = 0) -> np.ndarray:
        out = np.zeros(self.n_levels, dtype=np.int64)
        _check("pa_energy_hist", lib().pa_energy_hist(self._h, t, pop, _p(out, ctypes.c_int64), out.size))
        return out

    def q_hist(self, t: int) -> np.ndarray:
        out = np.zeros(self.q_bins, dtype=np.int64)
        _check("pa_q_hist", lib().pa_q_hist(self._h, t, _p(out, ctypes.c_int64), out.size))
        return out

    def family_hist(self, pop: int = 0):
        n = ctypes.c_int64()
        lib().pa_family_hist(self._h, pop, 0, None, None, ctypes.byref(n))
        eta = np.zeros(max(n.value, 1), dtype=np.int64)
        m = np.zeros(max(n.value, 1), dtype=np.int64)
        _check("pa_family_hist", lib().pa_family_hist(self._h, pop, eta.size, _p(eta, ctypes.c_int64),
                                                      _p(m, ctypes.c_int64), ctypes.byref(n)))
        return eta[:n.value].copy(), m[:n.value].copy()

    def size(self, pop: int = 0) -> int:
        n = ctypes.c_int64()
        _check("pa_population_size", lib().pa_population_size(self._h, pop, ctypes.byref(n)))
        return n.value

    def replicas(self, pop: int = 0, first: int = 0, n: Optional[int] = None):
        """(spins [n, N] int8, labels int32, energies int32) of slots first..first+n."""
        if n is None:
            n = self.size(pop) - first
        s = np.zeros((n, self.N), dtype=np.int8)
        lab = np.zeros(n, dtype=np.int32)
        E = np.zeros(n, dtype=np.int32)
        _check("pa_get_replicas", lib().pa_get_replicas(self._h, pop, first, n, _p(s, ctypes.c_int8),
                                                        _p(lab, ctypes.c_int32), _p(E, ctypes.c_int32)))
        return s, lab, E

    def population(self, pop: int = 0):
        """(spins [R~, N] int8, labels int32, energies): int32 energies for +-1
        couplings, int64 energies in units of 2^-20 for Gaussian ones."""
        if getattr(self, "model", 0) == PA_MODEL_GAUSS:
            n = self.size(pop)
            s = np.zeros((n, self.N), dtype=np.int8)
            lab = np.zeros(n, dtype=np.int32)
            _check("pa_get_replicas", lib().pa_get_replicas(self._h, pop, 0, n, _p(s, ctypes.c_int8),
                                                            _p(lab, ctypes.c_int32), None))
            return s, lab, self.genergies(pop)
        return self.replicas(pop, 0, None)

    # ---- Gaussian couplings
    def gobs(self, t: int, pop: int = 0) -> dict:
        o = GObs()
        _check("pa_gobservables", lib().pa_gobservables(self._h, t, pop, ctypes.byref(o)))
        return o.as_dict()

    def genergies(self, pop: int = 0) -> np.ndarray:
        n = self.size(pop)
        E = np.zeros(max(n, 1), dtype=np.int64)
        if n:
            _check("pa_get_genergies", lib().pa_get_genergies(self._h, pop, 0, n, _p(E, ctypes.c_int64)))
        return E[:n]

    def ql_hist(self, t: int) -> np.ndarray:
        out = np.zeros(self.q_bins, dtype=np.int64)
        _check("pa_ql_hist", lib().pa_ql_hist(self._h, t, _p(out, ctypes.c_int64), out.size))
        return out

    def gcouplings(self) -> np.ndarray:
        out = np.zeros(3 * self.N, dtype=np.int32)
        _check("pa_get_gcouplings", lib().pa_get_gcouplings(self._h, _p(out, ctypes.c_int32), out.size))
        return out

    def sweep_plan(self) -> dict:
        """The sweep launches of this run: the tile shape's index in ``sweep_shapes(L)``
        and, when the last wave of tiles runs as a second launch of smaller tiles, that
        shape's index and the first slot it covers (else -1 and 0)."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check("pa_sweep_plan", lib().pa_sweep_plan(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"shape": a.value, "tail_shape": b.value, "tail_from": c.value}

    def copy_counts(self, pop: int = 0) -> np.ndarray:
        n = ctypes.c_int64()
        lib().pa_get_copy_counts(self._h, pop, None, 0, ctypes.byref(n))
        out = np.zeros(max(n.value, 1), dtype=np.int32)
        _check("pa_get_copy_counts", lib().pa_get_copy_counts(self._h, pop, _p(out, ctypes.c_int32), out.size,
                                                              ctypes.byref(n)))
        return out[:n.value].copy()

    def parents(self, pop: int = 0) -> np.ndarray:
        n = ctypes.c_int64()
        lib().pa_get_parents(self._h, pop, None, 0, ctypes.byref(n))
        out = np.zeros(max(n.value, 1), dtype=np.int32)
        _check("pa_get_parents", lib().pa_get_parents(self._h, pop, _p(out, ctypes.c_int32), out.size,
                                                      ctypes.byref(n)))
        return out[:n.value].copy()

    def couplings(self) -> np.ndarray:
        J = np.zeros(3 * self.N, dtype=np.int8)
        _check("pa_get_couplings", lib().pa_get_couplings(self._h, _p(J, ctypes.c_int8), J.size))
        return J


class Shard:
    """One rank's share of a population annealing run split across ranks (pa_shard):
    the exchanges between the phases of a step go over torch.distributed (a process
    group of n_ranks ranks, gloo or any backend with CPU send/recv), all ranks call
    every method together.  ``local`` is this rank's run (its slots of the current
    population) for the per-rank readers (population, copy_counts)."""

    def __init__(self, L: int, R: int, disorder_seed: int, run_seed: int, betas, *, n_sweeps: int = 10,
                 sweeps_per_step=None, n_pop: int = 1, q_bins: int = 65, R_cap: int = 0, group=None, stream=None):
        import torch
        import torch.distributed as dist

        self.L, self.N, self.n_pop, self.q_bins = L, L ** 3, n_pop, q_bins
        self.rank, self.n_ranks = dist.get_rank(group), dist.get_world_size(group)
        self._holder = _ConfigHolder(L, R, disorder_seed, run_seed, betas, n_sweeps=n_sweeps,
                                     sweeps_per_step=sweeps_per_step, n_pop=n_pop, q_bins=q_bins, R_cap=R_cap)
        self._failure = None

        def guard(fn):
            def wrapped(*args):
                try:
                    fn(*args)
                    return 0
                except Exception as e:  # reported by the library as a failed step
                    self._failure = e
                    return 1
            return wrapped

        def allreduce(_, ptr, n):
            a = np.ctypeslib.as_array(ptr, shape=(n,))
            x = torch.from_numpy(a.copy())
            dist.all_reduce(x, group=group)
            a[:] = x.numpy()

        def allgather(_, ptr, n, out):
            x = torch.from_numpy(np.ctypeslib.as_array(ptr, shape=(n,)).copy())
            parts = [torch.zeros_like(x) for _ in range(self.n_ranks)]
            dist.all_gather(parts, x, group=group)
            np.ctypeslib.as_array(out, shape=(n * self.n_ranks,))[:] = torch.cat(parts).numpy()

        def send(_, dst, buf, nbytes):
            x = torch.from_numpy(np.ctypeslib.as_array(ctypes.cast(buf, ctypes.POINTER(ctypes.c_uint8)),
                                                       shape=(nbytes,)).copy())
            dist.send(x, dst, group=group)

        def recv(_, src, buf, nbytes):
            x = torch.zeros(nbytes, dtype=torch.uint8)
            dist.recv(x, src, group=group)
            ctypes.memmove(buf, x.numpy().ctypes.data, nbytes)

        self._callbacks = (_ALLREDUCE(guard(allreduce)), _ALLGATHER(guard(allgather)), _XFER(guard(send)),
                           _XFER(guard(recv)))
        self._comm = Comm(None, *self._callbacks)
        h = _vp()
        rc = lib().pa_shard_create(ctypes.byref(self._holder.cfg), self.rank, self.n_ranks, ctypes.byref(self._comm),
                                   _stream_handle(stream), ctypes.byref(h))
        self._raise_failure()
        _check("pa_shard_create", rc)
        self._h = h
        loc = _vp()
        _check("pa_shard_local", lib().pa_shard_local(self._h, ctypes.byref(loc)))
        self.local = Run._borrowed(loc, self, L, n_pop, q_bins)

    def _raise_failure(self):
        if self._failure is not None:
            e, self._failure = self._failure, None
            raise RuntimeError(f"host exchange failed: {e!r}") from e

    def step(self) -> int:
        rc = lib().pa_shard_step(self._h)
        self._raise_failure()
        return _check("pa_shard_step", rc)

    def run(self) -> None:
        while self.step() == 0:
            pass

    @property
    def t(self) -> int:
        return self.local.t

    def obs(self, t: int, pop: int = 0) -> dict:
        o = Obs()
        _check("pa_shard_observables", lib().pa_shard_observables(self._h, t, pop, ctypes.byref(o)))
        return o.as_dict()

    def extent(self, pop: int = 0):
        """(global slot of this rank's first slot, global population size)."""
        lo, R = ctypes.c_int64(), ctypes.c_int64()
        _check("pa_shard_extent", lib().pa_shard_extent(self._h, pop, ctypes.byref(lo), ctypes.byref(R)))
        return lo.value, R.value

    def q_hist(self, t: int) -> np.ndarray:
        out = np.zeros(self.q_bins, dtype=np.int64)
        _check("pa_shard_q_hist", lib().pa_shard_q_hist(self._h, t, _p(out, ctypes.c_int64), out.size))
        return out

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().pa_shard_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
