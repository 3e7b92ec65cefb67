"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point declared in include/lrbms.h, and the binding
refuses to run without it."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lrbms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lrbms_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("lrbms_offline_load", "lrbms_step", "lrbms_run", "lrbms_create", "lrbms_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1405_2810_gb300 import build
    lib_path = build.build()
    import ctypes
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1405_2810_gb300 import lrbms
    assert set(lrbms.EXPORTED) >= set(declared_symbols()), set(declared_symbols()) - set(lrbms.EXPORTED)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1405_2810_gb300 import lrbms
    monkeypatch.setattr(lrbms, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(lrbms, "_lib", None)
    with pytest.raises(RuntimeError):
        lrbms.library()


def test_create_rejects_bad_config():
    from paper_1405_2810_gb300 import lrbms
    with pytest.raises(lrbms.LrbmsError) as ei:
        lrbms.lrbms_create(max_slots=0)
    assert ei.value.code == lrbms.LRBMS_E_ARG
    for kw in (dict(refactor_stages=-1), dict(refactor_period=4, refactor_stages=5),
               dict(refactor_stages=9)):  # more stages than steps in the (default 8) period
        with pytest.raises(lrbms.LrbmsError) as ei:
            lrbms.lrbms_create(solver=lrbms.LRBMS_SOLVE_MIXED, **kw)
        assert ei.value.code == lrbms.LRBMS_E_ARG


def test_config_struct_matches_header():
    """The binding's lrbms_config fields are the header's, in the header's order."""
    from paper_1405_2810_gb300 import lrbms
    src = open(os.path.join(ROOT, "include", "lrbms.h")).read()
    body = re.search(r"typedef struct \{([^{}]*?)\} lrbms_config;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = [re.findall(r"(\w+)\s*$", decl.strip())[0] for decl in body.split(";") if decl.strip()]
    assert names == [f[0] for f in lrbms.Config._fields_]
