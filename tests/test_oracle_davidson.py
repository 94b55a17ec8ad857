"""Pins of the block-Davidson oracle (Sec. 2.4, Appendix A).

Each pin compares the oracle's step with something it does not compute
itself: a brute-force eigen-decomposition of the whole operator matrix (the
step is exact once the subspace spans the space), textbook special cases
(triangular and Hermitian matrices), the closed-form eigenvalues of the
homogeneous electron gas, and the Payne factor's algebraic values.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import biortho as BO
from oracle import davidson as DV
from oracle import operator as OP
from paper_2302_07420_gb300 import synth
from test_oracle_heg import closed_forms, heg_case


def _rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _phase_align(ref, got):
    """got_i * conj(phase of <ref_i|got_i>) for every row i."""
    ov = np.einsum("...i,...i->...", np.conj(ref), got)
    return got * (np.conj(ov) / np.abs(ov))[..., None]


# ---------------------------------------------------------------- Payne factor
def test_payne_values_and_limits():
    assert DV.payne(0.0) == 1.0
    assert DV.payne(1.0) == pytest.approx(65.0 / 81.0, abs=1e-15)
    assert DV.payne(0.5) == pytest.approx(40.0 / 41.0, abs=1e-15)   # 27+9+3+1 = 40 over 40 + 1
    x = np.linspace(0.0, 50.0, 2001)
    p = DV.payne(x)
    assert np.all(np.diff(p) < 0) and np.all(p > 0) and np.all(p <= 1)
    big = np.array([1e3, 1e4, 1e5])
    np.testing.assert_allclose(DV.payne(big) * 2 * big, 1.0, rtol=2e-3)   # -> 1/(2x)


def test_payne_argument_is_the_kinetic_energy_ratio_of_the_trial_vector():
    """Sec. 2.4: x(G) = |k+G|^2/2 divided by the trial vector's own kinetic energy sum |k+G'|^2/2 |v(G')|^2.

    For a trial vector that is one plane wave G0 that energy is t(G0), so the new direction is
    P(t(G)/t(G0)) (h v - eps v), with eps = h(G0, G0) and no component along G0 (the residual has none
    and P(1) keeps it zero); for a two-wave vector (a e_0 + b e_2)/norm it is (0.3 |a|^2 + 0.7 |b|^2)/norm^2."""
    rng = np.random.default_rng(41)
    t = np.array([0.3, 0.0, 0.7, 1.9, 4.2, 2.5])
    H = _rand_c(rng, 6, 6)
    v = np.zeros((1, 6), complex)
    v[0, 0] = 1.0
    kept, idx = DV.new_directions(v, v @ H.T, t)
    assert idx == [0]
    r = H[:, 0] - H[0, 0] * v[0]
    want = DV.payne(t / 0.3) * r
    want /= np.linalg.norm(want)
    np.testing.assert_allclose(_phase_align(want[None], kept[0][None])[0], want, atol=1e-13)
    # two plane waves: kinetic energy (0.3 * 1 + 0.7 * 4) / 5 = 0.62
    v = np.zeros((1, 6), complex)
    v[0, 0], v[0, 2] = 1.0 / np.sqrt(5.0), 2.0 / np.sqrt(5.0)
    kept, _ = DV.new_directions(v, v @ H.T, t)
    hv = v[0] @ H.T
    u = DV.payne(t / 0.62) * (hv - np.vdot(v[0], hv) * v[0])
    u -= np.vdot(v[0], u) * v[0]
    u /= np.linalg.norm(u)
    np.testing.assert_allclose(_phase_align(u[None], kept[0][None])[0], u, atol=1e-13)


@pytest.mark.parametrize("eps,kept", [(1e-6, True), (1e-11, False)])
def test_norm_cut_of_new_directions(eps, kept):
    """Sec. 2.4: a new direction whose norm after orthogonalisation is below 1e-8 is left out, one above
    it is kept.  h = diag(t) + eps X with v = e_0 leaves a residual of norm ~eps (P is 0.6-0.8 here)."""
    rng = np.random.default_rng(43)
    t = np.array([0.5, 0.55, 0.6, 0.7, 0.8])
    X = _rand_c(rng, 5, 5)
    H = np.diag(t).astype(complex) + eps * X
    v = np.zeros((1, 5), complex)
    v[0, 0] = 1.0
    new, _ = DV.new_directions(v, v @ H.T, t)
    nrm = np.linalg.norm(DV.payne(t / 0.5) * (H[:, 0] - H[0, 0] * v[0]))
    assert (1e-7 < nrm < 1e-4) if kept else (nrm < 1e-9)
    assert len(new) == (1 if kept else 0)


# ---------------------------------------------------------------- eigen-decomposition
def test_eig_sorted_equations_and_order():
    rng = np.random.default_rng(1)
    M = _rand_c(rng, 7, 7)
    lam, y, z = DV.eig_sorted(M)
    assert np.all(np.diff(lam.real) >= 0)
    np.testing.assert_allclose(M @ y, y * lam[None], atol=1e-12)
    np.testing.assert_allclose(z.conj().T @ M, lam[:, None] * z.conj().T, atol=1e-12)
    np.testing.assert_allclose(z.conj().T @ y, np.eye(7), atol=1e-12)


def test_eig_sorted_triangular_and_hermitian_cases():
    rng = np.random.default_rng(2)
    U = np.triu(_rand_c(rng, 6, 6))
    lam, _, _ = DV.eig_sorted(U)
    d = np.diag(U)
    np.testing.assert_allclose(lam, d[np.argsort(d.real)], atol=1e-12)   # triangular: the diagonal
    A = _rand_c(rng, 6, 6)
    Hm = A + A.conj().T
    lam, y, z = DV.eig_sorted(Hm)
    np.testing.assert_allclose(lam.real, np.linalg.eigvalsh(Hm), atol=1e-12)
    assert np.abs(lam.imag).max() < 1e-12
    np.testing.assert_allclose(z, y, atol=1e-12)                          # Hermitian: left = right


def test_appendix_a_gram_schmidt_keeps_the_diagonal():
    """GS of the eigenvectors: eps = phi^H h phi is upper triangular with the eigenvalues on the diagonal."""
    rng = np.random.default_rng(3)
    H = np.diag(np.arange(8.0)) + 0.4 * _rand_c(rng, 8, 8)
    lam, y, _ = DV.eig_sorted(H)
    phi = BO.gram_schmidt(y.T)                       # rows
    eps = np.conj(phi) @ H @ phi.T
    np.testing.assert_allclose(np.diag(eps), lam, atol=1e-12)
    assert np.abs(np.tril(eps, -1)).max() < 1e-12
    assert np.abs(np.triu(eps, 1)).max() > 1e-3      # non-Hermitian: not diagonal


# ---------------------------------------------------------------- dense step
def _dense_case(seed, n, m):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.2, 6.0, n))
    H = np.diag(t) + 0.3 * _rand_c(rng, n, n)
    v = BO.gram_schmidt(_rand_c(rng, m, n))
    return H, v, t


def _brute(H, m):
    """Lowest m right/left eigenvectors of H, made orthonormal / biorthonormal (rows)."""
    lam, y, z = DV.eig_sorted(H)
    phi, chi = BO.biorthonormalize(y[:, :m].T[None], z[:, :m].T[None])
    return lam[:m], phi[0], chi[0]


@pytest.mark.parametrize("n,m", [(6, 3), (7, 4), (5, 3)])
def test_dense_step_is_exact_when_the_subspace_is_the_space(n, m):
    H, v, t = _dense_case(10 + n, n, m)
    lam, phi, chi, d = DV.davidson_dense(H, v, t)
    assert d == n                                    # 2m - n new directions dropped as dependent
    lam_b, phi_b, chi_b = _brute(H, m)
    np.testing.assert_allclose(lam, lam_b, atol=1e-11)
    np.testing.assert_allclose(_phase_align(phi_b, phi), phi_b, atol=1e-10)
    np.testing.assert_allclose(_phase_align(phi_b, chi), chi_b, atol=1e-10)


def test_dense_invariant_subspace_is_kept():
    n, m = 9, 3
    H, _, t = _dense_case(21, n, m)
    lam_b, phi_b, chi_b = _brute(H, m)
    lam, phi, chi, d = DV.davidson_dense(H, phi_b, t)
    # only the first residual vanishes: for a non-normal h, h v_i - eps_ii v_i lies in span(v_0..v_i)
    # but is not zero, and the preconditioner takes it out of that span
    assert d == 2 * m - 1
    np.testing.assert_allclose(lam, lam_b, atol=1e-12)
    np.testing.assert_allclose(_phase_align(phi_b, phi), phi_b, atol=1e-10)
    # chi are left solutions of h compressed to the subspace, not of h itself: biorthonormal to phi,
    # and <chi_i|h|phi_j> upper triangular with the eigenvalues on the diagonal
    np.testing.assert_allclose(np.conj(chi) @ phi.T, np.eye(m), atol=1e-12)
    eps = np.conj(chi) @ H @ phi.T
    np.testing.assert_allclose(np.diag(eps), lam_b, atol=1e-11)
    assert np.abs(np.tril(eps, -1)).max() < 1e-11


def test_dense_step_improves_the_lowest_eigenvalues():
    """The Ritz values approach the exact ones from a rough start (a plausible-mistake net: a wrong
    sign in the residual or a transposed subspace matrix loses this)."""
    n, m = 40, 4
    rng = np.random.default_rng(31)
    t = np.sort(rng.uniform(0.2, 20.0, n))            # a kinetic-like diagonal with a weak non-Hermitian part
    H = np.diag(t) + 0.05 * _rand_c(rng, n, n)
    lam_b, phi_b, _ = _brute(H, m)
    v = BO.gram_schmidt(phi_b + 0.05 * _rand_c(rng, m, n))
    e0 = np.abs(np.diag(np.conj(v) @ H @ v.T) - lam_b).max()
    lam, phi, _, d = DV.davidson_dense(H, v, t)
    assert d == 2 * m
    assert np.abs(lam - lam_b).max() < 0.02 * e0


# ---------------------------------------------------------------- TC operator
def _tc_case(seed, kmesh, ecut, m, nocc):
    p = synth.tiny_params(seed, kmesh=kmesh, fft=(8, 9, 10), ecut=ecut, nbands=m, nocc=nocc)
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 600 + seed, [S.kpG(k) for k in range(S.Nk)],
                                         S.npw_max, m, perturb=0.1)
    occ = np.zeros((S.Nk, m))
    occ[:, :nocc] = [1.0, 0.7][:nocc]
    return S, c_phi, c_chi, occ


def _dense_tc(S, c_phi, c_chi, occ):
    """The operator matrix on each sphere, column by column (h on unit vectors)."""
    e = np.zeros((S.Nk, S.npw_max, S.npw_max), dtype=np.complex128)
    for k in range(S.Nk):
        e[k, np.arange(S.npw[k]), np.arange(S.npw[k])] = 1.0
    he = DV.h_apply(S, c_phi, c_chi, occ, e)
    return [he[k, : S.npw[k], : S.npw[k]].T for k in range(S.Nk)]   # H[k][:, j] = h e_j


def test_h_on_an_empty_band_equals_the_operator_output():
    S, c_phi, c_chi, occ = _tc_case(3, (1, 1, 2), 1.2, 3, 2)
    hv = DV.h_apply(S, c_phi, c_chi, occ, c_phi)
    out = OP.total(OP.apply_operator(S, c_phi, c_chi, occ)) + OP.kinetic_coeffs(S, c_phi)
    np.testing.assert_allclose(hv, out, atol=1e-13 * np.abs(out).max())


def test_tc_step_is_exact_on_a_small_sphere():
    """npw <= 2m: the step returns the brute-force eigenpairs of the whole TC operator matrix."""
    m = 4
    S, c_phi, c_chi, occ = _tc_case(4, (1, 1, 1), 0.8, m, 2)
    n = S.npw[0]
    assert m < n <= 2 * m
    Hd = _dense_tc(S, c_phi, c_chi, occ)
    phi, chi, lam, d = DV.davidson_step(S, c_phi, c_chi, occ)
    assert d[0] == n
    lam_b, phi_b, chi_b = _brute(Hd[0], m)
    np.testing.assert_allclose(lam[0], lam_b, atol=1e-11 * np.abs(lam_b).max())
    np.testing.assert_allclose(_phase_align(phi_b, phi[0, :, :n]), phi_b, atol=1e-9)
    np.testing.assert_allclose(_phase_align(phi_b, chi[0, :, :n]), chi_b, atol=1e-9)


def test_tc_step_appendix_a_on_the_outputs():
    """Outputs: phi orthonormal, chi biorthonormal; <phi_i|h|phi_j> and <chi_i|h|phi_j> upper
    triangular with the Ritz values on the diagonal (Appendix A applied to the projected h)."""
    S, c_phi, c_chi, occ = _tc_case(5, (1, 1, 2), 1.2, 3, 2)
    phi, chi, lam, d = DV.davidson_step(S, c_phi, c_chi, occ)
    assert np.all(d == 6)
    hphi = DV.h_apply(S, c_phi, c_chi, occ, phi)
    for k in range(S.Nk):
        np.testing.assert_allclose(np.conj(phi[k]) @ phi[k].T, np.eye(3), atol=1e-12)
        np.testing.assert_allclose(np.conj(chi[k]) @ phi[k].T, np.eye(3), atol=1e-12)
        sc = np.abs(lam[k]).max()
        for bra in (phi[k], chi[k]):
            eps = np.conj(bra) @ hphi[k].T
            np.testing.assert_allclose(np.diag(eps), lam[k], atol=1e-11 * sc)
            assert np.abs(np.tril(eps, -1)).max() < 1e-11 * sc
    # the Ritz values are those of the brute-force projected operator on span(v, w)
    Hd = _dense_tc(S, c_phi, c_chi, occ)
    for k in range(S.Nk):
        assert np.all(lam[k].real >= np.sort(np.linalg.eigvals(Hd[k]).real)[:3].min() - 1e-9)


@pytest.mark.parametrize("case", [dict(nelec=14, rs=4.0, fft=16, radius2=16, radius2_occ=1),
                                  dict(nelec=38, rs=2.5, fft=15, radius2=9, radius2_occ=2)])
def test_heg_plane_waves_are_fixed_points(case):
    """Plane waves diagonalise the HEG TC operator: no new direction, closed-form eigenvalues."""
    S, c, occ = heg_case(**case)
    idx, e = closed_forms(S, c)
    G = S.miller[0][idx] @ S.B
    ref = 0.5 * np.einsum("ij,ij->i", G, G) + sum(e[t] for t in OP.TERMS)
    phi, chi, lam, d = DV.davidson_step(S, c, c, occ)
    m = c.shape[1]
    assert d[0] == m
    np.testing.assert_allclose(np.sort(lam[0].real), np.sort(ref.real), atol=1e-11 * np.abs(ref).max())
    assert np.abs(lam[0].imag).max() < 1e-11 * np.abs(ref).max()
    # same span as the input plane waves; chi = phi (BITC = TC for plane waves)
    P_in = c[0].T @ np.conj(c[0])
    P_out = phi[0].T @ np.conj(phi[0])
    np.testing.assert_allclose(P_out, P_in, atol=1e-10)
    np.testing.assert_allclose(chi[0], phi[0], atol=1e-9)
