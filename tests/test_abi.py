"""CPU-only: the C-ABI library loads and exports every entry point that
include/a2dmrg.h declares (no compute call is made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:a2_status|const char\*)\s+(a2_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for n in ["a2_ctx_create", "a2_tt_create", "a2_mpo_load", "a2_additive_sweep",
              "a2_coarse_solve", "a2_energy", "a2_heff_apply"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2505_23429_gb300 import build
    lib = build.build(verbose=False)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (a2_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    import ctypes
    dll = ctypes.CDLL(lib)
    for n in _declared():
        assert hasattr(dll, n)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2505_23429_gb300.a2dmrg as b
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        b.lib()
