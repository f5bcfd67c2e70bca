"""The C ABI library builds, loads and exports every entry point include/pa.h
declares; the Python binding covers them all.  No compute calls (CPU only)."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(pa_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def palib():
    from paper_1711_02146_gb300 import build, pa
    build.build()
    return pa.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pa_create", "pa_step", "pa_run", "pa_observables", "pa_destroy", "pa_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(palib):
    for name in declared_functions():
        assert hasattr(palib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1711_02146_gb300 import pa
    assert set(declared_functions()) <= set(pa.SIGNATURES)


def test_strerror_without_gpu(palib):
    from paper_1711_02146_gb300 import pa
    assert pa.strerror(pa.PA_ERR_CAPACITY).startswith("population exceeded")
    assert pa.strerror(0) == "ok"


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    from paper_1711_02146_gb300 import pa
    monkeypatch.setattr(pa, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pa, "_lib", None)
    with pytest.raises(ImportError):
        pa.lib()


def _up(n):
    return (n + 255) // 256 * 256


def test_footprint_is_the_slab_layout_without_gpu(palib):
    """pa_footprint is host-only and gives the exact size of the run's one device
    allocation: every buffer of the +-1 layout rounded up to 256 bytes, one
    Boltzmann weight table per distinct temperature increment (one table for the
    adaptive schedule)."""
    import numpy as np
    from paper_1711_02146_gb300 import pa
    from paper_1711_02146_gb300.workloads import Workload, linear_betas
    step_rec = 88
    for L, R, n_pop, betas in [(4, 1000, 1, linear_betas(51, 5.0)), (10, 123457, 2, np.array([0.0, 0.1, 0.2, 0.25])),
                               (6, 7, 1, None)]:
        w = Workload("fp", L=L, R=R, disorder_seed=1, run_seed=2, betas=betas, n_temps=0 if betas is not None else 40,
                     eps_target=0.0 if betas is not None else 0.2, n_pop=n_pop)
        N, T, Rc = L ** 3, (len(betas) if betas is not None else 40), w.capacity
        pitch, nlev = -(-Rc // 1024) * 1024, 3 * L ** 3 + 1
        ncb, nfs = -(-Rc // 1024), math.isqrt(2 * Rc) + 2
        want = _up(3 * N) + _up(16 * N) + _up(4) + _up(8 * T * 65)
        per_pop = (2 * (_up(N * pitch) + _up(4 * pitch)) + 3 * _up(4 * pitch) + _up(4 * ncb) + _up(8 * ncb) + _up(4)
                   + _up(4 * T * nlev) + 2 * _up(4 * nlev) + 2 * _up(4 * (Rc + 1)) + _up(4 * nfs) + _up(8)
                   + _up(step_rec * T))
        want += n_pop * per_pop
        n_tables = len({float(d).hex() for d in np.diff(betas)}) if betas is not None else 1
        want += _up(8 * n_tables * nlev)
        assert pa.footprint(w) == want, (L, R, n_pop)
    # Gaussian couplings: energies, weights and their fixed-order partial sums (the
    # chunk totals of 256 slots, then every tree level but the last), copy-number
    # tables, moment partials and records; per-step site and weight tables instead of
    # the +-1 weight tables
    grec, kpat, kgw = 64, 64, 16384
    for L, R, T in [(4, 1000, 11), (6, 300_000, 5)]:
        w = Workload("g", L=L, R=R, disorder_seed=1, run_seed=2, betas=linear_betas(T, 2.0), model=1)
        N, Rc = L ** 3, w.capacity
        pitch, nlev = -(-Rc // 1024) * 1024, 3 * N + 1
        ncb, nchunk, nmb, nfs = -(-Rc // 1024), -(-Rc // 256), -(-Rc // 4096), math.isqrt(2 * Rc) + 2
        levels, m = nchunk, nchunk
        while m > 256:
            m = -(-m // 256)
            levels += m
        want = _up(3 * N) + _up(16 * N) + _up(4) + _up(8 * T * 65)
        want += (2 * (_up(N * pitch) + _up(4 * pitch)) + 3 * _up(4 * pitch) + _up(4 * ncb) + _up(8 * ncb) + _up(4)
                 + _up(4 * T * nlev) + 2 * _up(4 * nlev) + 2 * _up(4 * (Rc + 1)) + _up(4 * nfs) + _up(8)
                 + _up(step_rec * T))
        want += (_up(8 * pitch) + _up(8 * Rc) + _up(8 * levels) + 2 * _up(4 * Rc) + _up(16 * nmb) + _up(grec * T))
        want += _up(12 * N) + _up(4 * T * N * kpat) + _up(8 * T * kgw) + _up(8 * T * 65)
        assert pa.footprint(w) == want, (L, R)
