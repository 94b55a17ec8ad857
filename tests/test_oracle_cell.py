"""Pins of the oracle's basis and divergence-correction constant (Sec. 2.5)."""
import numpy as np
import pytest

from conftest import make_setup
from oracle import cell as CL
from oracle import ewald
from paper_2302_07420_gb300 import synth

# Madelung constant of the simple-cubic lattice of unit charges in a neutralising
# background: v_M L = -2.837297479480620 (standard value, e.g. Nijboer & De Wette 1957).
SC_MADELUNG = 2.837297479480620


def test_simple_cubic_madelung_constant():
    for L in (1.0, 15.54052, 7.67663317071):
        g0 = CL.gamma0(np.eye(3) * L, (1, 1, 1), CL.default_alpha(np.eye(3) * L, (1, 1, 1)))
        cC = 4 * np.pi * g0 / L ** 3
        assert abs(cC * L - SC_MADELUNG) < 2e-12


@pytest.mark.parametrize("kmesh", [(1, 1, 1), (2, 2, 2), (4, 4, 4), (1, 2, 3)])
def test_correction_constant_is_minus_supercell_madelung(kmesh):
    p = synth.si_params(kmesh=kmesh)
    lat = p["lattice"]
    Om = abs(np.linalg.det(lat))
    g0 = CL.gamma0(lat, kmesh, CL.default_alpha(lat, kmesh))
    vM = ewald.madelung(lat * np.asarray(kmesh)[:, None])
    assert abs(4 * np.pi * g0 / Om + vM) < 1e-10 * abs(vM)


def test_triclinic_and_alpha_insensitivity():
    p = synth.tiny_params(0)
    lat, km = p["lattice"], (2, 1, 3)
    Om = abs(np.linalg.det(lat))
    a0 = CL.default_alpha(lat, km)
    c1 = 4 * np.pi * CL.gamma0(lat, km, a0) / Om
    c2 = 4 * np.pi * CL.gamma0(lat, km, a0 * (12 / 14) ** 2) / Om
    assert abs(c1 - c2) < 1e-10 * abs(c1)
    assert abs(c1 + ewald.madelung(lat * np.asarray(km)[:, None])) < 1e-10 * abs(c1)


def test_sphere_counts_and_order():
    # |n|^2 <= 16 holds 257 integer vectors (Gauss lattice-point count for r^2 = 16)
    S = make_setup(synth.heg_params(14, 4.0, 16, 16))
    assert S.npw.tolist() == [257]
    m = S.miller[0]
    assert all(tuple(m[i]) < tuple(m[i + 1]) for i in range(len(m) - 1))
    # |n|^2 <= 5 holds 57 vectors (1 + 6 + 12 + 8 + 6 + 24)
    S = make_setup(synth.heg_params(114, 2.0, 48, 144))
    assert int(np.sum(np.einsum("ij,ij->i", S.miller[0], S.miller[0]) <= 5)) == 57
    # the sphere is invariant under k -> k + G: counts depend only on the k-point class
    S = make_setup(synth.si_params())
    assert S.npw.sum() == sum(len(CL.sphere_miller(S.kcart[k] + S.B[0], S.B, S.ecut)) for k in range(S.Nk))


def test_sphere_cutoff_is_inclusive():
    """A plane wave exactly on the cutoff belongs to the sphere (|k+G|^2/2 <= E_cut).  On the simple-cubic
    cell of edge 2 pi (b_i = unit vectors, so |G|^2 = |m|^2 exactly in floating point) at Gamma, the sphere
    of E_cut = r2/2 holds the integer vectors with |m|^2 <= r2: the cumulative sums of r3(n), the number of
    representations of n as a sum of three squares (1, 6, 12, 8, 6, 24, 24, 0, 12, 30 for n = 0..9)."""
    counts = {1: 7, 2: 19, 3: 27, 4: 33, 5: 57, 6: 81, 7: 81, 8: 93, 9: 123}
    B = CL.reciprocal(2.0 * np.pi * np.eye(3))
    assert np.array_equal(B, np.eye(3))
    for r2, want in counts.items():
        assert len(CL.sphere_miller(np.zeros(3), B, 0.5 * r2)) == want, r2


def test_alpha_reading_on_the_fcc_supercell():
    """sqrt(alpha) = L_min/12 with L_min the shortest vector of the Born-von Karman supercell: for the
    fcc cell (|a_i| = a/sqrt 2) on an n x n x n mesh that is n a/sqrt 2 (the supercell is the fcc cell
    scaled by n), on a 4 x 2 x 1 mesh the shortest of 4 a_1, 2 a_2, a_3 and their combinations, a/sqrt 2."""
    lat = synth.si_params()["lattice"]
    a = 10.26
    for n in (1, 2, 4):
        assert abs(CL.default_alpha(lat, (n, n, n)) - (n * a / np.sqrt(2.0) / 12.0) ** 2) < 1e-12
    assert abs(CL.default_alpha(lat, (4, 2, 1)) - (a / np.sqrt(2.0) / 12.0) ** 2) < 1e-12


def test_kmesh_and_box_conventions():
    f = CL.kmesh_frac((4, 1, 3))
    assert f.shape == (12, 3)
    assert np.all(f > -0.5) and np.all(f <= 0.5)
    assert CL.fft_rep(6).tolist() == [0, 1, 2, -3, -2, -1]
    assert CL.fft_rep(5).tolist() == [0, 1, 2, -2, -1]


def test_heg_cell_from_rs():
    """HEG geometry (Sec. 4, homogeneous electron gas): four electrons in the simple-cubic cell of
    a = 7.67663317071 bohr have r_s = 3 bohr, i.e. a = (4 pi N / 3)^(1/3) r_s; the same rule gives the 14- and
    114-electron cells of the HEG workloads."""
    p = synth.heg_params(4, 3.0, 16, 4)
    assert abs(p["lattice"][0, 0] - 7.67663317071) < 1e-10
    assert np.count_nonzero(p["lattice"] - np.diag(np.diag(p["lattice"]))) == 0
    Omega = abs(np.linalg.det(p["lattice"]))
    assert abs((3 * Omega / (4 * np.pi * 4)) ** (1 / 3) - 3.0) < 1e-12
    assert abs(synth.WORKLOADS["heg_14"]()["lattice"][0, 0] - 15.54052) < 1e-5
