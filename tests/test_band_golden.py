"""The stored band-point values (tests/golden/si_k444_band.json, written by make_golden.py from oracle/
only) regenerate from their seeds, and the library's host band constants and layout reproduce them.

The stored operator outputs at the band point are the parity reference for a CUDA band-point path.
"""
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "golden", "si_k444_band.json")


@pytest.fixture(scope="module")
def golden():
    if not os.path.exists(PATH):
        pytest.skip("si_k444_band.json not written")
    return json.load(open(PATH))


def test_band_inputs_regenerate(golden):
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden as MG
    p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ = MG.band_inputs()
    assert golden["k_band_frac"] == MG.K_BAND
    assert int(SB.npw[S.Nk]) == golden["npw_band"]
    np.testing.assert_array_equal(SB.miller[S.Nk], np.array(golden["miller_band"]))
    phi = np.array(golden["input_probe"]["phi"]).view(complex).ravel()
    chi = np.array(golden["input_probe"]["chi"]).view(complex).ravel()
    assert np.abs(b_phi[0, :, 5] - phi).max() < 1e-15 and np.abs(b_chi[0, :, 5] - chi).max() < 1e-15
    assert abs(SB.gamma_b[0] - golden["gamma_b"]) < 1e-13 * abs(golden["gamma_b"])
    np.testing.assert_allclose(SB.W[0], golden["W"], rtol=0, atol=1e-13)
    out_r = np.array(golden["out_R"]).view(complex).reshape(S.nbands, -1)
    assert out_r.shape[1] == golden["npw_band"] and np.abs(out_r).max() > 1e-3


def test_library_band_constants_and_layout_reproduce_the_stored_values(golden):
    from paper_2302_07420_gb300 import build as B
    if not os.path.exists(B.LIB):
        pytest.skip("libtc.so not built")
    from paper_2302_07420_gb300 import _lib, synth
    from paper_2302_07420_gb300.operator import band_constants, band_layout
    _lib._lib = None
    p = synth.si_params()
    args = (p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"])
    g, W = band_constants(*args, np.array(golden["k_band_frac"]))
    assert abs(g[0] - golden["gamma_b"]) < 1e-12 * abs(golden["gamma_b"])
    np.testing.assert_allclose(W[0], golden["W"], rtol=0, atol=1e-11 * np.abs(golden["W"]).max())
    npw, miller = band_layout(*args, np.array(golden["k_band_frac"]))
    assert npw[0] == golden["npw_band"]
    np.testing.assert_array_equal(miller[0, : npw[0]], np.array(golden["miller_band"]))
