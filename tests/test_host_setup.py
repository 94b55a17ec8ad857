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
from oracle import band as BD
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
    npw_max = int(x[o]); o += 1
    npw = x[o:o + Nk].astype(int); o += Nk
    miller = x[o:o + Nk * npw_max * 3].astype(int).reshape(Nk, npw_max, 3); o += Nk * npw_max * 3
    box = x[o:o + Nk * npw_max].astype(int).reshape(Nk, npw_max); o += Nk * npw_max
    deriv = []
    for _ in range(4):
        d = {}
        for key, size, shape in (("tabV", nd * 2 * N, (nd, 2, N)), ("tabU", nd * 2 * N, (nd, 2, N)),
                                 ("hartV", 2 * N, (2, N)), ("hartU", N, (N,)), ("hartUs", 2 * N, (2, N))):
            d[key] = x[o:o + size].reshape(shape); o += size
        d["corr"], d["amp"] = x[o:o + 2], x[o + 2:o + 4]; o += 4
        deriv.append(d)
    gsq0 = x[o]; o += 1
    band = dict(found=bool(x[o]), gamma_b=x[o + 1], W=x[o + 2:o + 5]); o += 5
    assert o == len(x)
    return dict(Omega=Om, alpha=al, Gamma0=G0, corr=(c0, c1), Nk=Nk, did=did, delta=delta, tabV=tabV, tabU=tabU,
                hartV=hartV, hartU=hartU, hartUs=hartUs, npw_max=npw_max, npw=npw, miller=miller, box=box,
                deriv=deriv, gsq0=gsq0, band=band)


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
    _compare_tables(T, S, KN.JastrowKernels(S.A, S.C))


def _compare_tables(T, S, ks):
    """Exchange and Hartree-type tables of the probe (T) against the oracle's kernels with kernel data ks."""
    c_phi = np.zeros((S.Nk, S.nbands, S.npw_max), complex)
    right = OP.TCOperator(S, c_phi, c_phi, np.zeros((S.Nk, S.nbands)), left=False, kset=ks)
    left = OP.TCOperator(S, c_phi, c_phi, np.zeros((S.Nk, S.nbands)), left=True, kset=ks)
    P = S.Gbox.reshape(-1, 3)
    for ko in range(S.Nk):
        for kp in range(S.Nk):
            i = T["did"][ko, kp]
            np.testing.assert_allclose(T["delta"][i], S.kcart[ko] - S.kcart[kp], rtol=0, atol=1e-14)
            KR, KL = right.kern(ko, kp), left.kern(ko, kp)
            sc = max(np.abs(KR["V"]).max(), 1e-300)
            np.testing.assert_allclose(T["tabV"][i, 0], KR["V"].ravel(), rtol=0, atol=1e-13 * sc)
            np.testing.assert_allclose(T["tabV"][i, 1], KL["V"].ravel(), rtol=0, atol=1e-13 * sc)
            p = T["delta"][i][None, :] + P
            for s in range(2):
                U = np.stack([KR["U"][s][d].ravel() for d in range(3)], axis=-1)       # i p u~/Omega
                lib = 1j * p * T["tabU"][i, s][:, None]
                np.testing.assert_allclose(lib, U, rtol=0, atol=1e-13 * max(np.abs(U).max(), 1e-30))
    VhR, UhR, usR = right.hartree_kernels()
    VhL, _, _ = left.hartree_kernels()
    sc = max(np.abs(VhR).max(), 1e-300)
    np.testing.assert_allclose(T["hartV"][0], VhR.ravel(), rtol=0, atol=1e-13 * sc)
    np.testing.assert_allclose(T["hartV"][1], VhL.ravel(), rtol=0, atol=1e-13 * sc)
    for s in range(2):
        np.testing.assert_allclose(T["hartUs"][s], usR[s].ravel(), rtol=0,
                                   atol=1e-13 * max(np.abs(usR[s]).max(), 1e-300))
    np.testing.assert_allclose(T["hartU"], (usR[0] + usR[1]).ravel() / S.Omega, rtol=0,
                               atol=1e-13 * max(np.abs(T["hartU"]).max(), 1e-300))


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_derivative_tables_match_the_oracle(probe, tmp_path, name):
    """The tables of dK/dA_s and dK/dC_s (kernel_data modes KD_DA_PP .. KD_DC_AP, which the adjoint uses)
    against the oracle's closed-form derivatives (oracle/kernels.py, pinned against differences of the
    kernels), including the correction coefficients and amplitudes; the Coulomb part and the other
    channel carry no derivative."""
    p = CASES[name]()
    if name.startswith("heg"):      # unequal channels, so that a channel mix-up shows
        p["A"], p["C"] = [p["A"][0], 1.3 * p["A"][1]], [p["C"][0], 0.8 * p["C"][1]]
    T = _run(probe, tmp_path, p, div=1, uf=2.0)
    S = make_setup(p, div_correction=1, ushort_factor=2.0)
    for mode, (wrt, s0) in enumerate((("A", 0), ("A", 1), ("C", 0), ("C", 1))):
        ks = KN.JastrowKernels(S.A, S.C, deriv=(wrt, s0))
        D = dict(T["deriv"][mode], did=T["did"], delta=T["delta"])
        _compare_tables(D, S, ks)
        for s in range(2):
            ref = ks.corr(s, S.Gamma0, S.ushort_factor, S.Nk)
            assert abs(D["corr"][s] - ref) <= 1e-12 * max(abs(ref), 1e-30), (mode, s, D["corr"][s], ref)
            assert D["amp"][s] == ks.amp(s), (mode, s)
    assert abs(T["gsq0"] - KN.gradu_sq(np.array([0.0]), S.A[0], S.C[0])[0]) <= 1e-15 * abs(T["gsq0"])


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_layout_and_band_constants_match_the_oracle(probe, tmp_path, name):
    """Sphere sizes, Miller vectors (lexicographic, zero padded) and box indices (-1 padded) of every
    k-point, and Gamma_b and W at an off-mesh k, against the oracle (oracle/cell.py, oracle/band.py)."""
    p = CASES[name]()
    T = _run(probe, tmp_path, p)
    S = make_setup(p)
    assert T["npw_max"] == S.npw_max and T["npw"].tolist() == S.npw.tolist()
    n = S.n[0]
    for k in range(S.Nk):
        m = S.npw[k]
        assert np.array_equal(T["miller"][k, :m], S.miller[k])
        assert not T["miller"][k, m:].any() and np.all(T["box"][k, m:] == -1)
        i0, i1, i2 = S.box_index[k]
        assert np.array_equal(T["box"][k, :m], (i0 * n + i1) * n + i2)
    kc = np.array([0.13, 0.27, -0.31]) @ S.B
    assert T["band"]["found"]
    gb = BD.gamma_band(S.lattice, S.kmesh, S.alpha, kc)
    W = BD.aux_vector_sum(S.lattice, S.kmesh, S.alpha, kc)
    assert abs(T["band"]["gamma_b"] - gb) <= 1e-12 * abs(gb)
    np.testing.assert_allclose(T["band"]["W"], W, rtol=0, atol=1e-12 * np.abs(W).max())


def test_host_sphere_cutoff_and_box_fit(probe, tmp_path):
    """On the simple-cubic cell of edge 2 pi at Gamma (b_i = unit vectors exactly) the sphere of
    E_cut = r2/2 holds the integer vectors with |m|^2 <= r2 (cumulative sums of r3(n); a wave on the
    cutoff belongs to the sphere), and a sphere that reaches Miller index n/2 of an even box (which the
    box index n/2 cannot tell from -n/2) is refused."""
    counts = {1: 7, 2: 19, 3: 27, 5: 57, 9: 123, 25: 515}
    base = dict(lattice=2.0 * np.pi * np.eye(3), kmesh=(1, 1, 1), fft=(12,) * 3, nbands=1, nocc=1,
                A=[1.0, 1.0], C=[1.0, 1.0])
    for r2, want in counts.items():
        T = _run(probe, tmp_path, dict(base, ecut=0.5 * r2))
        assert T["npw"].tolist() == [want], r2
    out = str(tmp_path / "refused.bin")
    p = dict(base, ecut=0.5 * 36)      # |m| = 6 = n/2 on the axes
    args = [probe, out] + ["%.17g" % x for x in np.asarray(p["lattice"]).ravel()] + ["1", "1", "1"]
    args += ["%.17g" % p["ecut"], "12", "1", "1", "1", "1", "1", "1", "0", "1", "1"]
    r = subprocess.run(args, capture_output=True, text=True)
    assert r.returncode == 1 and "does not fit" in r.stderr


def _refused(probe, tmp_path, p, **kw):
    args = [probe, str(tmp_path / "refused.bin")] + ["%.17g" % x for x in np.asarray(p["lattice"]).ravel()]
    args += [str(k) for k in p["kmesh"]] + ["%.17g" % p["ecut"], str(p["fft"][0]), str(p["nbands"]), str(p["nocc"])]
    args += ["%.17g" % x for x in p["A"]] + ["%.17g" % x for x in p["C"]] + ["0", "1", "1"]
    r = subprocess.run(args, capture_output=True, text=True)
    return r.returncode, r.stderr.strip()


@pytest.mark.parametrize("change,message", [
    (dict(fft=(10, 10, 10)), "unsupported: FFT box size"),
    (dict(kmesh=(0, 1, 1)), "kmesh entries must be in [1, 16]"),
    (dict(kmesh=(17, 1, 1)), "kmesh entries must be in [1, 16]"),
    (dict(nocc=0), "need 0 < nocc <= nbands"),
    (dict(nocc=4, nbands=3), "need 0 < nocc <= nbands"),
    (dict(ecut=0.0), "ecut_ha must be positive"),
    (dict(C=[1.0, 0.0]), "Jastrow C must be positive"),
    (dict(A=[-0.1, 1.0]), "Jastrow A must be non-negative"),
    (dict(lattice=np.zeros((3, 3))), "lattice is singular"),
    (dict(ecut=40.0), "plane-wave sphere does not fit the FFT box"),
])
def test_host_setup_refuses_invalid_parameters(probe, tmp_path, change, message):
    """The argument checks of tc_init's host setup, each with its message (and nothing built)."""
    p = dict(synth.tiny_params(3, kmesh=(1, 1, 2), fft=(9, 9, 9), ecut=1.6, scale=5.0), **change)
    rc, err = _refused(probe, tmp_path, p)
    assert rc == 1 and err.startswith(message), (rc, err)


def test_host_setup_accepts_the_limits(probe, tmp_path):
    """The edges of the accepted ranges: A = 0 (the Hartree-Fock limit), nocc = nbands, a 16-point mesh axis."""
    p = dict(synth.tiny_params(3, kmesh=(16, 1, 1), fft=(9, 9, 9), ecut=1.6, scale=5.0), A=[0.0, 0.0])
    p["nocc"] = p["nbands"]
    T = _run(probe, tmp_path, p)
    assert T["Nk"] == 16
