"""The C-ABI library builds, loads without a GPU and exports every symbol of include/tc.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:tc_status|const char\s*\*)\s+(tc_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_07420_gb300 import _lib
    from paper_2302_07420_gb300 import build as B
    srcs = [os.path.join(B.SRC, f) for f in os.listdir(B.SRC)] + [os.path.join(ROOT, "include", "tc.h")]
    if not os.path.exists(B.LIB) or os.path.getmtime(B.LIB) < max(os.path.getmtime(s) for s in srcs):
        if not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available")
        B.build()
    _lib._lib = None
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("tc_init", "tc_apply", "tc_energy", "tc_layout", "tc_destroy", "tc_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2302_07420_gb300 import _lib
    names = _declared()
    assert sorted(_lib.EXPORTED) == names
    for n in names:
        assert hasattr(lib, n), n


def test_init_error_paths_without_gpu(lib):
    """Invalid parameters are rejected by the host setup before any device call."""
    import ctypes
    from paper_2302_07420_gb300 import _lib, synth
    p = synth.tiny_params(0, kmesh=(1, 1, 2), fft=(10, 10, 10), ecut=1.6, scale=5.0)
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], 3, 2, p["A"], p["C"])
    h = ctypes.c_void_p()
    assert lib.tc_init(ctypes.byref(prm), ctypes.byref(h)) == _lib.TC_ERR_UNSUPPORTED
    assert b"box" in lib.tc_last_error(None)
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], (9, 9, 9), 3, 4, p["A"], p["C"])
    assert lib.tc_init(ctypes.byref(prm), ctypes.byref(h)) == _lib.TC_ERR_ARG
    assert lib.tc_init(None, ctypes.byref(h)) == _lib.TC_ERR_ARG
    assert lib.tc_destroy(None) == _lib.TC_ERR_STATE


def test_alu_peak_argument_errors_without_gpu(lib):
    """tc_alu_peak checks its arguments before any device call."""
    import ctypes
    from paper_2302_07420_gb300 import _lib
    out = ctypes.c_double(0.0)
    assert lib.tc_alu_peak(7, 50.0, ctypes.byref(out), None) == _lib.TC_ERR_ARG
    assert lib.tc_alu_peak(_lib.TC_FP32, 0.0, ctypes.byref(out), None) == _lib.TC_ERR_ARG
    assert lib.tc_alu_peak(_lib.TC_FP64, 5000.0, ctypes.byref(out), None) == _lib.TC_ERR_ARG
    assert lib.tc_alu_peak(_lib.TC_FP32, 50.0, None, None) == _lib.TC_ERR_ARG
    assert b"tc_alu_peak" in lib.tc_last_error(None)


def test_injected_allocation_fault_without_gpu(lib, monkeypatch):
    """TC_FAULT=alloc: tc_init fails with TC_ERR_OOM after the host setup, before any device call."""
    import ctypes
    from paper_2302_07420_gb300 import _lib, synth
    p = synth.tiny_params(0, kmesh=(1, 1, 2), fft=(9, 9, 9), ecut=1.6, scale=5.0)
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], 3, 2, p["A"], p["C"])
    h = ctypes.c_void_p()
    monkeypatch.setenv("TC_FAULT", "alloc")
    assert lib.tc_init(ctypes.byref(prm), ctypes.byref(h)) == _lib.TC_ERR_OOM
    assert b"TC_FAULT=alloc" in lib.tc_last_error(None)
    assert not h.value
    bad = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], (10, 10, 10), 3, 2, p["A"], p["C"])
    assert lib.tc_init(ctypes.byref(bad), ctypes.byref(h)) == _lib.TC_ERR_UNSUPPORTED   # setup errors first


def test_precision_modes_without_gpu(lib):
    """TC_FP32_COMP (compensated accumulation, not built) is refused as unsupported by the host
    setup; an unknown precision is an argument error; TC_BF16_STORE passes the setup (TC_FAULT=alloc
    stops it before any device call)."""
    import ctypes
    from paper_2302_07420_gb300 import _lib, synth
    p = synth.tiny_params(0, kmesh=(1, 1, 2), fft=(9, 9, 9), ecut=1.6, scale=5.0)
    h = ctypes.c_void_p()
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], 3, 2, p["A"], p["C"], precision="fp32_comp")
    assert lib.tc_init(ctypes.byref(prm), ctypes.byref(h)) == _lib.TC_ERR_UNSUPPORTED
    assert b"TC_FP32_COMP" in lib.tc_last_error(None)
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], 3, 2, p["A"], p["C"], precision=9)
    assert lib.tc_init(ctypes.byref(prm), ctypes.byref(h)) == _lib.TC_ERR_ARG
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], 3, 2, p["A"], p["C"], precision="bf16_store")
    import os as _os
    old = _os.environ.get("TC_FAULT")
    _os.environ["TC_FAULT"] = "alloc"
    try:
        assert lib.tc_init(ctypes.byref(prm), ctypes.byref(h)) == _lib.TC_ERR_OOM
    finally:
        if old is None:
            del _os.environ["TC_FAULT"]
        else:
            _os.environ["TC_FAULT"] = old
