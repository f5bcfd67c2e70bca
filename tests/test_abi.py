"""The C ABI library builds, loads and exports every entry point include/pa.h
declares; the Python binding covers them all.  No compute calls (CPU only)."""
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
