"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point declared in include/ra.h (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ra.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ra_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ra_problem_create", "ra_eval_dual", "ra_solve", "ra_recover_primal",
                 "ra_init_prices", "ra_problem_destroy", "ra_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2104_00282_gb300 import build as B
    path = B.build()
    L = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    L.ra_version.restype = ctypes.c_char_p
    assert b"sm_103a" in L.ra_version()
    L.ra_status_string.restype = ctypes.c_char_p
    assert L.ra_status_string(4) == b"not converged"


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    from paper_2104_00282_gb300 import ra
    monkeypatch.setattr(ra, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(ra, "_lib", None)
    try:
        ra.lib()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("binding loaded a library that does not exist")
