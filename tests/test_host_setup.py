"""The library's FP64 host tables (csrc/tc_setup.cpp) against the oracle's kernels, on the CPU.

A small probe (tests/host/setup_probe.cpp) is compiled with the library's own setup source and writes
the tables it builds: V_2a and V_2a^dagger and u~_pp, u~_ap at k_out - k_part + G for every distinct
k-point difference (with the G = 0 rules and the correction constant), the Hartree-type tables and the
3a2/3b6 correction scalars.  They must equal the oracle's values (oracle/operator.py ``kern`` and
``hartree_kernels``, oracle/kernels.py) to FP64 rounding.  No GPU is involved.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import make_setup
from oracle import kernels as KN
from oracle import operator as OP
from paper_2302_07420_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_07420_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("probe") / "setup_probe")
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(ROOT, "tests", "host", "setup_probe.cpp"), os.path.join(CSRC, "tc_setup.cpp")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _run(probe, tmp_path, p, div=1, uf=1.0, alpha=0.0):
    out = str(tmp_path / "tables.bin")
    args = [probe, out] + ["%.17g" % x for x in np.asarray(p["lattice"]).ravel()] + [str(k) for k in p["kmesh"]]
    args += ["%.17g" % p["ecut"], str(p["fft"][0]), str(p["nbands"]), str(p["nocc"])]
    args += ["%.17g" % x for x in p["A"]] + ["%.17g" % x for x in p["C"]] + ["%.17g" % alpha, str(div), "%.17g" % uf]
    r = subprocess.run(args, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    x = np.fromfile(out, dtype=np.float64)
    Om, al, G0, nd, c0, c1, Nk, N = x[:8]
    nd, Nk, N = int(nd), int(Nk), int(N)
    o = 8
    did = x[o:o + Nk * Nk].astype(int).reshape(Nk, Nk); o += Nk * Nk
    delta = x[o:o + 3 * nd].reshape(nd, 3); o += 3 * nd
    tabV = x[o:o + nd * 2 * N].reshape(nd, 2, N); o += nd * 2 * N
    tabU = x[o:o + nd * 2 * N].reshape(nd, 2, N); o += nd * 2 * N
    hartV = x[o:o + 2 * N].reshape(2, N); o += 2 * N
    hartU = x[o:o + N]; o += N
    hartUs = x[o:o + 2 * N].reshape(2, N); o += 2 * N
    assert o == len(x)
    return dict(Omega=Om, alpha=al, Gamma0=G0, corr=(c0, c1), Nk=Nk, did=did, delta=delta, tabV=tabV, tabU=tabU,
                hartV=hartV, hartU=hartU, hartUs=hartUs)


CASES = {
    "si_k222_12": lambda: synth.si_params(kmesh=(2, 2, 2), fft=12, ecut=1.5),
    "triclinic_k112_9": lambda: synth.tiny_params(3, kmesh=(1, 1, 2), fft=(9, 9, 9), ecut=1.6, scale=5.0),
    "heg_14_16": lambda: synth.WORKLOADS["heg_14"](),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("div,uf", [(1, 1.0), (0, 1.0), (1, 2.0)])
def test_host_tables_match_the_oracle(probe, tmp_path, name, div, uf):
    p = CASES[name]()
    T = _run(probe, tmp_path, p, div=div, uf=uf)
    S = make_setup(p, div_correction=div, ushort_factor=uf)
    assert T["Nk"] == S.Nk
    assert abs(T["Omega"] - S.Omega) < 1e-13 * S.Omega
    assert abs(T["alpha"] - S.alpha) < 1e-14 * S.alpha
    assert abs(T["Gamma0"] - S.Gamma0) < 1e-12 * abs(S.Gamma0)
    ks = KN.JastrowKernels(S.A, S.C)
    for s in range(2):
        ref = ks.corr(s, S.Gamma0, S.ushort_factor, S.Nk)
        assert abs(T["corr"][s] - ref) < 1e-12 * max(abs(ref), 1e-30), (s, T["corr"][s], ref)
    c_phi = np.zeros((S.Nk, S.nbands, S.npw_max), complex)
    right = OP.TCOperator(S, c_phi, c_phi, np.zeros((S.Nk, S.nbands)), left=False)
    left = OP.TCOperator(S, c_phi, c_phi, np.zeros((S.Nk, S.nbands)), left=True)
    P = S.Gbox.reshape(-1, 3)
    for ko in range(S.Nk):
        for kp in range(S.Nk):
            i = T["did"][ko, kp]
            np.testing.assert_allclose(T["delta"][i], S.kcart[ko] - S.kcart[kp], rtol=0, atol=1e-14)
            KR, KL = right.kern(ko, kp), left.kern(ko, kp)
            sc = np.abs(KR["V"]).max()
            np.testing.assert_allclose(T["tabV"][i, 0], KR["V"].ravel(), rtol=0, atol=1e-13 * sc)
            np.testing.assert_allclose(T["tabV"][i, 1], KL["V"].ravel(), rtol=0, atol=1e-13 * sc)
            p = T["delta"][i][None, :] + P
            for s in range(2):
                U = np.stack([KR["U"][s][d].ravel() for d in range(3)], axis=-1)       # i p u~/Omega
                lib = 1j * p * T["tabU"][i, s][:, None]
                np.testing.assert_allclose(lib, U, rtol=0, atol=1e-13 * max(np.abs(U).max(), 1e-30))
    VhR, UhR, usR = right.hartree_kernels()
    VhL, _, _ = left.hartree_kernels()
    sc = np.abs(VhR).max()
    np.testing.assert_allclose(T["hartV"][0], VhR.ravel(), rtol=0, atol=1e-13 * sc)
    np.testing.assert_allclose(T["hartV"][1], VhL.ravel(), rtol=0, atol=1e-13 * sc)
    for s in range(2):
        np.testing.assert_allclose(T["hartUs"][s], usR[s].ravel(), rtol=0, atol=1e-13 * np.abs(usR[s]).max())
    np.testing.assert_allclose(T["hartU"], (usR[0] + usR[1]).ravel() / S.Omega, rtol=0,
                               atol=1e-13 * np.abs(T["hartU"]).max())
