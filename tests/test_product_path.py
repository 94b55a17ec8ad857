"""The product path (the package and its C library) has no CPU fallback and never touches the oracle."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2302_07420_gb300")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2302_07420_gb300 import _lib, synth
    from paper_2302_07420_gb300.operator import Context
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libtc.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()
    p = synth.tiny_params(0)
    with pytest.raises(RuntimeError, match="not built"):
        Context(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"])


def test_package_imports_no_oracle():
    code = ("import sys; import paper_2302_07420_gb300, paper_2302_07420_gb300.operator, "
            "paper_2302_07420_gb300.autograd, paper_2302_07420_gb300.synth; "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "sys.exit(1 if bad else 0)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr


def test_product_sources_do_not_name_the_oracle():
    pat = re.compile(r"^\s*(from|import)\s+oracle\b|\boracle[/\\]", re.M)
    for dirpath, _, files in os.walk(PKG):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".hpp", ".h")):
                src = open(os.path.join(dirpath, f), encoding="utf-8").read()
                assert not pat.search(src), f
