"""Structural pins of the oracle on random cells (P5, P6, P7, P8, c18).

Odd FFT boxes are used: there every Miller integer has a unique symmetric
representative, so the discrete operator keeps the exchange and adjoint
symmetries of the continuum one exactly (aliasing included).
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import operator as OP
from paper_2302_07420_gb300 import synth


def case(seed=0, kmesh=(1, 1, 2), fft=(9, 9, 11), ecut=1.6, nbands=3, nocc=2, fill=(1.0, 1.0), **kw):
    p = synth.tiny_params(seed, kmesh=kmesh, fft=fft, ecut=ecut, nbands=nbands, nocc=nocc, scale=5.0)
    S = make_setup(p, **kw)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 60 + seed, [S.kpG(k) for k in range(S.Nk)],
                                         S.npw_max, S.nbands, perturb=0.15)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, :nocc] = np.asarray(fill)[None, :nocc]
    return S, c_phi, c_chi, occ


@pytest.mark.parametrize("div", [1, 0])
def test_adjointness(div):
    """<chi_i | h phi_j> = <h^dagger chi_i | phi_j> for all i, j at every k (P6)."""
    S, c_phi, c_chi, occ = case(seed=1, fill=(1.0, 0.6), div_correction=div)
    out_r, out_l = OP.tc_apply(S, c_phi, c_chi, occ)
    for k in range(S.Nk):
        lhs = np.conj(c_chi[k]) @ out_r[k].T          # [i, j] = <chi_i| h phi_j>
        rhs = np.conj(out_l[k]) @ c_phi[k].T          # [i, j] = <h^dag chi_i| phi_j>
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13 * np.abs(lhs).max())


def test_biorthogonal_gauge():
    """Phi -> Phi M, X -> X M^-dagger (per k, within equal-occupation blocks) (P5)."""
    S, c_phi, c_chi, occ = case(seed=2)
    rng = np.random.default_rng(7)
    out_r, out_l = OP.tc_apply(S, c_phi, c_chi, occ)
    E0 = OP.energy_terms(S, c_phi, c_chi, occ)["total"]
    Ms = []
    p2, x2 = np.zeros_like(c_phi), np.zeros_like(c_chi)
    for k in range(S.Nk):
        M = np.eye(S.nbands, dtype=complex)
        no = S.nocc
        M[:no, :no] += 0.4 * (rng.standard_normal((no, no)) + 1j * rng.standard_normal((no, no)))
        M[no:, no:] *= 0.7 * np.exp(0.3j)
        Ms.append(M)
        # columns are orbitals: Phi' = Phi M, X' = X M^{-H}; here rows are orbitals
        p2[k] = M.T @ c_phi[k]
        x2[k] = np.linalg.inv(M).conj() @ c_chi[k]
    r2, l2 = OP.tc_apply(S, p2, x2, occ)
    for k in range(S.Nk):
        M = Ms[k]
        np.testing.assert_allclose(r2[k], M.T @ out_r[k], rtol=0, atol=1e-12 * np.abs(out_r).max())
        np.testing.assert_allclose(l2[k], np.linalg.inv(M).conj() @ out_l[k], rtol=0,
                                   atol=1e-12 * np.abs(out_l).max())
    E1 = OP.energy_terms(S, p2, x2, occ)["total"]
    assert abs(E1 - E0) < 1e-12 * abs(E0)


def test_translation_covariance():
    """c(G) -> c(G) e^{-i(k+G).t} for a grid translation t: outputs follow, E is invariant (P7)."""
    S, c_phi, c_chi, occ = case(seed=3)
    t = (2 / S.n[0]) * S.lattice[0] - (3 / S.n[1]) * S.lattice[1] + (4 / S.n[2]) * S.lattice[2]
    ph = np.zeros((S.Nk, S.npw_max), dtype=complex)
    for k in range(S.Nk):
        ph[k, : S.npw[k]] = np.exp(-1j * S.kpG(k) @ t)
    out_r, out_l = OP.tc_apply(S, c_phi, c_chi, occ)
    r2, l2 = OP.tc_apply(S, c_phi * ph[:, None], c_chi * ph[:, None], occ)
    np.testing.assert_allclose(r2, out_r * ph[:, None], rtol=0, atol=1e-12 * np.abs(out_r).max())
    np.testing.assert_allclose(l2, out_l * ph[:, None], rtol=0, atol=1e-12 * np.abs(out_l).max())
    E0 = OP.energy_terms(S, c_phi, c_chi, occ)["total"]
    E1 = OP.energy_terms(S, c_phi * ph[:, None], c_chi * ph[:, None], occ)["total"]
    assert abs(E1 - E0) < 1e-12 * abs(E0)


def test_energy_quadratic_in_A():
    """At fixed C, E(A) = E0 + E1 A + E2 A^2 exactly, corrections included (P8)."""
    S, c_phi, c_chi, occ = case(seed=4)
    C = S.C.copy()
    As = [0.3, 0.9, 1.4, 2.2]
    Es = []
    for a in As:
        Sa = make_setup(synth.tiny_params(4, kmesh=(1, 1, 2), fft=(9, 9, 11), ecut=1.6, scale=5.0),
                        A=[a, a], C=C)
        Es.append(OP.energy_terms(Sa, c_phi, c_chi, occ)["total"])
    coef = np.polyfit(As[:3], Es[:3], 2)
    assert abs(np.polyval(coef, As[3]) - Es[3]) < 1e-11 * abs(Es[3])


def _deriv(fun, h):
    """Exact derivative at 0 of a polynomial of degree <= 4 from a 4-point stencil."""
    return (8 * (fun(h) - fun(-h)) - (fun(2 * h) - fun(-2 * h))) / (12 * h)


def test_energy_gradient_is_the_operator():
    """dE/dchi^* = f (T + h) phi and dE/dphi^* = f (T + h^dagger) chi, corrections off (c18).

    E is a polynomial of degree 3 along any orbital direction, so the stencil is exact.
    """
    S, c_phi, c_chi, occ = case(seed=5, fill=(1.0, 0.55), div_correction=0)
    rng = np.random.default_rng(11)
    out_r, out_l = OP.tc_apply(S, c_phi, c_chi, occ)
    gr = OP.kinetic_coeffs(S, c_phi) + out_r
    gl = OP.kinetic_coeffs(S, c_chi) + out_l
    mask = np.zeros((S.Nk, S.npw_max))
    for k in range(S.Nk):
        mask[k, : S.npw[k]] = 1.0
    for which in ("chi", "phi"):
        d = (rng.standard_normal(c_phi.shape) + 1j * rng.standard_normal(c_phi.shape)) * mask[:, None]
        if which == "chi":
            fun = lambda h: OP.energy_terms(S, c_phi, c_chi + h * d, occ)["total"]
            ref = 2.0 / S.Nk * np.real(np.sum(occ[:, :, None] * np.conj(d) * gr))
        else:
            fun = lambda h: OP.energy_terms(S, c_phi + h * d, c_chi, occ)["total"]
            ref = 2.0 / S.Nk * np.real(np.sum(occ[:, :, None] * np.conj(gl) * d))
        fd = _deriv(fun, 1e-2)
        assert abs(fd - ref) < 1e-10 * abs(ref), (which, fd, ref)


@pytest.mark.parametrize("term", OP.TERMS)
def test_pins_detect_a_planted_mistake(term, monkeypatch):
    """Scaling any single term by 1.3 must break the energy-gradient or adjoint identity."""
    orig = OP.TCOperator._apply_k

    def planted(self, k, terms):
        acc = orig(self, k, terms)
        if term in acc:
            acc[term] = 1.3 * acc[term]
        return acc

    S, c_phi, c_chi, occ = case(seed=5, fill=(1.0, 0.55), div_correction=0)
    monkeypatch.setattr(OP.TCOperator, "_apply_k", planted)
    out_r, out_l = OP.tc_apply(S, c_phi, c_chi, occ)
    gr = OP.kinetic_coeffs(S, c_phi) + out_r
    rng = np.random.default_rng(11)
    d = rng.standard_normal(c_phi.shape) + 1j * rng.standard_normal(c_phi.shape)
    for k in range(S.Nk):
        d[k, :, S.npw[k]:] = 0
    fun = lambda h: OP.energy_terms(S, c_phi, c_chi + h * d, occ)["total"]
    ref = 2.0 / S.Nk * np.real(np.sum(occ[:, :, None] * np.conj(d) * gr))
    grad_broken = abs(_deriv(fun, 1e-2) - ref) > 1e-8 * abs(ref)
    lhs = np.conj(c_chi[0]) @ out_r[0].T
    rhs = np.conj(out_l[0]) @ c_phi[0].T
    adj_broken = np.abs(lhs - rhs).max() > 1e-10 * np.abs(lhs).max()
    assert grad_broken or adj_broken


def test_partners_enter_only_through_the_density_matrix():
    """Density-matrix mixing (Sec. 2.4): partners enter the operator only through sum_q f_q phi_q chi_q^*.

    Splitting every partner into two identical copies with occupations beta f and (1 - beta) f
    leaves every output unchanged, divergence corrections (general-overlap forms) included.
    """
    p = synth.tiny_params(3, kmesh=(1, 1, 2), fft=(9, 9, 11), ecut=1.6, nbands=2, nocc=2, scale=5.0)
    S1 = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 77, [S1.kpG(k) for k in range(S1.Nk)], S1.npw_max, 2,
                                         perturb=0.1)
    occ1 = np.array([[1.0, 0.6]] * S1.Nk)
    r1, l1 = OP.tc_apply(S1, c_phi, c_chi, occ1)
    S2 = make_setup(p, nbands=4, nocc=4)
    beta = 0.3
    r2, l2 = OP.tc_apply(S2, np.concatenate([c_phi, c_phi], axis=1), np.concatenate([c_chi, c_chi], axis=1),
                         np.concatenate([beta * occ1, (1 - beta) * occ1], axis=1))
    scale = np.abs(r1).max()
    for half in (slice(0, 2), slice(2, 4)):
        np.testing.assert_allclose(r2[:, half], r1, rtol=0, atol=1e-13 * scale)
        np.testing.assert_allclose(l2[:, half], l1, rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("fft,ecut,exact", [((9, 9, 9), 1.6, True), ((12, 12, 12), 1.6, True),
                                            ((12, 12, 12), 6.0, False)])
def test_left_occupied_pair_fields_are_conjugates_of_the_right(fft, ecut, exact):
    """P_L(a, b) = conj P_R(b, a) (conj U(p) = U(-p) for U = i p u~): h6_L = conj h6_R and the two h3
    kinds swap under conjugation.  Exact on the grid for odd boxes and for pair densities clear of the
    Nyquist planes; an even box whose pair densities wrap onto them breaks it (the library then
    computes both sides)."""
    from paper_2302_07420_gb300 import synth as SY
    p = SY.tiny_params(3, kmesh=(1, 1, 2), fft=fft, ecut=ecut, nbands=3, nocc=2, scale=5.0)
    S = make_setup(p)
    c_phi, c_chi = SY.random_orbitals(SY.SEED0 + 903, [S.kpG(k) for k in range(S.Nk)], S.npw_max, 3,
                                      perturb=0.1)
    occ = np.zeros((S.Nk, 3))
    occ[:, :2] = [1.0, 0.7]
    R = OP.TCOperator(S, c_phi, c_chi, occ, left=False)
    L = OP.TCOperator(S, c_phi, c_chi, occ, left=True)
    R.prepare()
    L.prepare()
    err = max(np.abs(L.h6 - np.conj(R.h6)).max() / np.abs(R.h6).max(),
              max(np.abs(L.h3a4[k] - np.conj(R.h3b[k])).max() for k in range(S.Nk)) /
              max(np.abs(R.h3b[k]).max() for k in range(S.Nk)),
              max(np.abs(L.h3b[k] - np.conj(R.h3a4[k])).max() for k in range(S.Nk)) /
              max(np.abs(R.h3a4[k]).max() for k in range(S.Nk)))
    if exact:
        assert err < 1e-14
    else:
        assert err > 1e-9
