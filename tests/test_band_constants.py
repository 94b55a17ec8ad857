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


@pytest.mark.parametrize("case", ["si_k444", "triclinic_k112"])
def test_band_layout_matches_the_oracle_spheres(lib, case):
    from paper_2302_07420_gb300.operator import band_layout
    from conftest import make_setup
    if case.startswith("si"):
        p = synth.si_params()
    else:
        p = synth.tiny_params(3, kmesh=(1, 1, 2), fft=(9, 9, 9), ecut=1.6, scale=5.0)
    npw, miller = band_layout(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"],
                              POINTS)
    SB = BD.BandSetup(make_setup(p), POINTS)
    for i in range(len(POINTS)):
        ref = SB.miller[SB.Nk + i]
        assert npw[i] == len(ref)
        np.testing.assert_array_equal(miller[i, : npw[i]], ref)
        assert not miller[i, npw[i]:].any()


def test_band_layout_errors(lib):
    import ctypes
    from paper_2302_07420_gb300 import _lib
    p = synth.si_params(kmesh=(2, 2, 2))
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"])
    kf = np.ascontiguousarray(POINTS[:1])
    npw = np.zeros(1, dtype=np.int32)
    m = np.zeros((1, 4, 3), dtype=np.int32)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    assert lib.tc_band_layout(ctypes.byref(prm), kf.ctypes.data_as(dp), 1, 4, npw.ctypes.data_as(ip),
                              m.ctypes.data_as(ip)) == _lib.TC_ERR_ARG           # 4 < the sphere
    assert b"max_npw" in lib.tc_last_error(None)
    assert lib.tc_band_layout(ctypes.byref(prm), kf.ctypes.data_as(dp), 1, 0, npw.ctypes.data_as(ip),
                              None) == _lib.TC_OK and npw[0] > 4
    big = _lib.make_params(p["lattice"], p["kmesh"], 60.0, p["fft"], p["nbands"], p["nocc"], p["A"], p["C"])
    assert lib.tc_band_layout(ctypes.byref(big), kf.ctypes.data_as(dp), 1, 0, npw.ctypes.data_as(ip),
                              None) == _lib.TC_ERR_ARG                          # spheres overflow the box


def test_band_layout_at_mesh_points_is_the_mesh_layout(lib):
    """The library builds the SCF spheres with the same sphere rule: at the mesh points themselves the band
    layout equals the oracle's mesh spheres (all 64 k-points of the 4x4x4 workload)."""
    from paper_2302_07420_gb300.operator import band_layout
    from conftest import make_setup
    p = synth.si_params()
    S = make_setup(p)
    npw, miller = band_layout(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"],
                              S.kfrac)
    assert npw.tolist() == S.npw.tolist()
    for k in range(S.Nk):
        np.testing.assert_array_equal(miller[k, : npw[k]], S.miller[k])
