"""The seeded input recipes produce the stated workloads (CPU).

Constants: the FCC cell of a = 10.26 bohr (Omega = a^3/4), the HEG cells of N electrons at r_s
(L = (4 pi N/3)^(1/3) r_s), the Jastrow parameters of Eqs. A_normalize and cusp
(A = sqrt(Omega/(4 pi N)), C_pp = sqrt(2A), C_ap = sqrt(A)), the 256-cell batch's ranges, and the
biorthonormality of the random orbital sets.
"""
import collections

import numpy as np

from conftest import make_setup
from paper_2302_07420_gb300 import synth


def test_silicon_like_cell():
    p = synth.si_params()
    Om = abs(np.linalg.det(p["lattice"]))
    assert abs(Om - 10.26 ** 3 / 4) < 1e-9 and abs(Om - 270.0114) < 1e-4
    assert p["kmesh"] == (4, 4, 4) and p["fft"] == (24, 24, 24) and p["ecut"] == 7.5
    assert p["nbands"] == p["nocc"] == 4 and p["nelec"] == 8
    np.testing.assert_allclose(p["A"], [1.63886, 1.63886], atol=1e-5)
    np.testing.assert_allclose(p["C"], [1.81045, 1.28018], atol=1e-5)


def test_heg_cells():
    h14, h114 = synth.WORKLOADS["heg_14"](), synth.WORKLOADS["heg_114"]()
    assert abs(h14["lattice"][0, 0] - 15.54052) < 1e-5 and abs(h114["lattice"][0, 0] - 15.63248) < 1e-5
    np.testing.assert_allclose(h14["A"], [4.61880, 4.61880], atol=1e-5)
    np.testing.assert_allclose(h14["C"], [3.03934, 2.14914], atol=1e-5)
    np.testing.assert_allclose(h114["A"], [1.63299, 1.63299], atol=1e-5)
    np.testing.assert_allclose(h114["C"], [1.80720, 1.27789], atol=1e-5)
    assert (h14["nocc"], h114["nocc"]) == (7, 57) and (h14["fft"][0], h114["fft"][0]) == (16, 48)
    S = make_setup(h114)                               # sphere |n|^2 <= 144 on the 48^3 box
    assert max(np.abs(m).max() for m in S.miller) == 12


def test_heg_batch_ranges():
    cells = synth.heg_batch(256)
    assert len(cells) == 256
    assert {c["nelec"] for c in cells} == {14, 38, 54, 66}
    assert {c["fft"][0] for c in cells} == {16, 18, 20, 24, 25, 27, 30, 32}
    assert set(collections.Counter(c["kmesh"] for c in cells)) == {(1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2)}
    for c in cells:
        Om = abs(np.linalg.det(c["lattice"]))
        rs = (3 * Om / (4 * np.pi * c["nelec"])) ** (1 / 3)
        assert 1.0 <= rs <= 5.0
        assert c["nocc"] == c["nbands"] == c["nelec"] // 2
        A = np.sqrt(Om / (4 * np.pi * c["nelec"]))
        np.testing.assert_allclose(c["A"], [A, A], rtol=1e-12)
        np.testing.assert_allclose(c["C"], [np.sqrt(2 * A), np.sqrt(A)], rtol=1e-12)
    again = synth.heg_batch(256)[17]                   # seeded
    assert np.array_equal(again["lattice"], cells[17]["lattice"]) and again["kmesh"] == cells[17]["kmesh"]


def test_random_orbitals_are_biorthonormal():
    p = synth.si_params(kmesh=(2, 1, 1))
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 1, [S.kpG(k) for k in range(S.Nk)], S.npw_max, S.nbands)
    for k in range(S.Nk):
        n = S.npw[k]
        P, X = c_phi[k, :, :n], c_chi[k, :, :n]
        np.testing.assert_allclose(np.conj(X) @ P.T, np.eye(S.nbands), atol=1e-12)
        np.testing.assert_allclose(np.einsum("ij,ij->i", np.conj(P), P).real, 1.0, atol=1e-12)
        assert 1e-4 < np.abs(X - P).max() < 0.1          # the left set is the right set plus a small perturbation
        assert not c_phi[k, :, n:].any()
