"""The library's band-point constants (tc_band_constants, host only) against the oracle (oracle/band.py).

Both sides compute Gamma_b(k) = Omega/(4 sqrt(pi^3 alpha)) - (1/N_k) sum_{q,G} A_aux(k - q + G) and
W(k) = sum_{q,G} (k - q + G) A_aux(k - q + G) (Sec. 2.6.3 after Eq. divcorr_2ax_scf, Eq. correction_nabla)
independently; the oracle's values are themselves pinned by a phased Ewald sum (tests/test_oracle_band.py).
No GPU is needed: the call does no device work.
"""
import numpy as np
import pytest

from oracle import band as BD
from oracle import cell as CL
from paper_2302_07420_gb300 import synth

POINTS = np.array([[0.13, 0.27, -0.31], [0.5, 0.0, 0.125], [-0.07, 0.41, 0.33]])


@pytest.fixture(scope="module")
def lib():
    from paper_2302_07420_gb300 import _lib
    from paper_2302_07420_gb300 import build as B
    import os
    if not os.path.exists(B.LIB):
        if not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available")
        B.build()
    _lib._lib = None
    return _lib.load()


@pytest.mark.parametrize("case", ["si_k444", "si_k222", "triclinic_k112"])
def test_band_constants_match_the_oracle(lib, case):
    from paper_2302_07420_gb300.operator import band_constants
    if case.startswith("si"):
        p = synth.si_params(kmesh=(4, 4, 4) if case == "si_k444" else (2, 2, 2))
    else:
        p = synth.tiny_params(3, kmesh=(1, 1, 2), fft=(9, 9, 9), ecut=1.6, scale=5.0)
    g, W = band_constants(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"],
                          POINTS)
    B = CL.reciprocal(p["lattice"])
    a = CL.default_alpha(p["lattice"], p["kmesh"])
    for i, kf in enumerate(POINTS):
        k = kf @ B
        gr = BD.gamma_band(p["lattice"], p["kmesh"], a, k)
        Wr = BD.aux_vector_sum(p["lattice"], p["kmesh"], a, k)
        assert abs(g[i] - gr) < 1e-12 * abs(gr), (i, g[i], gr)
        assert np.abs(W[i] - Wr).max() < 1e-11 * max(np.abs(Wr).max(), 1e-3), (i, W[i], Wr)


def test_band_constants_errors(lib):
    import ctypes
    from paper_2302_07420_gb300 import _lib
    from paper_2302_07420_gb300.operator import band_constants
    p = synth.si_params(kmesh=(2, 2, 2))
    args = (p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"])
    for on_mesh in ([0.5, 0.0, 0.0], [0.0, 0.0, 0.0], [1.5, -1.0, 0.5]):
        with pytest.raises(_lib.TCError) as e:
            band_constants(*args, np.array(on_mesh))
        assert e.value.status == _lib.TC_ERR_ARG and "SCF mesh" in str(e.value)
    prm = _lib.make_params(*args)
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.tc_band_constants(ctypes.byref(prm), None, 1, None, None) == _lib.TC_ERR_ARG
    assert lib.tc_band_constants(ctypes.byref(prm), None, 0, None, None) == _lib.TC_OK
    assert lib.tc_band_constants(None, None, 0, None, None) == _lib.TC_ERR_ARG
