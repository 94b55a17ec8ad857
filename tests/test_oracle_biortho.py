"""Pins of oracle/biortho.py (Sec. 2.1 biorthogonal condition, Sec. 2.3 Gram-Schmidt)."""
import numpy as np

from oracle import biortho as BO


def _raw(seed, nk=3, nb=5, npw=40):
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((nk, nb, npw)) + 1j * rng.standard_normal((nk, nb, npw))
    chi = phi + 0.3 * (rng.standard_normal((nk, nb, npw)) + 1j * rng.standard_normal((nk, nb, npw)))
    phi[:, :, -4:] = 0.0   # zero padding beyond the sphere stays zero
    chi[:, :, -4:] = 0.0
    return phi, chi


def _proj(X):
    """Projector on the span of the rows of X."""
    Q, _ = np.linalg.qr(X.T)
    return Q @ np.conj(Q.T)


def test_biorthonormal_and_normalised():
    phi0, chi0 = _raw(1)
    phi, chi = BO.biorthonormalize(phi0, chi0)
    for k in range(phi.shape[0]):
        nb = phi.shape[1]
        np.testing.assert_allclose(np.conj(chi[k]) @ phi[k].T, np.eye(nb), atol=1e-13)
        np.testing.assert_allclose(np.conj(phi[k]) @ phi[k].T, np.eye(nb), atol=1e-13)
        # spans unchanged
        np.testing.assert_allclose(_proj(phi[k]), _proj(phi0[k]), atol=1e-12)
        np.testing.assert_allclose(_proj(chi[k]), _proj(chi0[k]), atol=1e-12)
    assert np.all(phi[:, :, -4:] == 0) and np.all(chi[:, :, -4:] == 0)


def test_idempotent():
    phi, chi = BO.biorthonormalize(*_raw(2))
    phi2, chi2 = BO.biorthonormalize(phi, chi)
    np.testing.assert_allclose(phi2, phi, atol=1e-13)
    np.testing.assert_allclose(chi2, chi, atol=1e-12)


def test_gram_schmidt_is_qr_up_to_phases():
    """Gram-Schmidt in band order = QR of the columns with a positive-real diagonal of R."""
    phi0, _ = _raw(3, nk=1)
    Q = BO.gram_schmidt(phi0[0])
    q, r = np.linalg.qr(phi0[0].T)
    ph = np.diag(r) / np.abs(np.diag(r))
    np.testing.assert_allclose(Q, (q * ph[None, :]).T, atol=1e-13)
