"""Biorthonormalisation of right and left orbitals per k-point (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.1 (the BITC paragraph): left and right orbitals obey the biorthogonal
condition <chi_i|phi_j> = delta_ij and the normalisation <phi_i|phi_i> = 1.
The library's helper produces such a pair from arbitrary inputs, per k-point,
in band order:

1. phi is orthonormalised by modified Gram-Schmidt (each band in turn minus its
   projections on the bands before it, then normalised), the orthonormalisation
   TC++ applies to its orbitals (Sec. 2.3);
2. chi' (the left input) is replaced by chi_j = sum_i chi'_i (M^-1)_ij with
   M_ij = <phi_i|chi'_j>, i.e. X = X' (Phi^H X')^-1 in column form, so that
   <chi_j|phi_l> = delta_jl and span(chi) = span(chi').

Coefficients are on the plane-wave sphere (zero padded); inner products are
sums over the sphere, <a|b> = sum_G conj(a(G)) b(G).

Parity pins (tests/test_oracle_biortho.py): chi^H phi = I and phi^H phi = I,
spans unchanged (projectors), idempotence, and Gram-Schmidt against numpy's QR.
"""
import numpy as np


def gram_schmidt(P):
    """Rows of P (nb, npw) orthonormalised in order (modified Gram-Schmidt)."""
    Q = np.array(P, dtype=np.complex128)
    for i in range(Q.shape[0]):
        for j in range(i):
            Q[i] -= np.vdot(Q[j], Q[i]) * Q[j]
        Q[i] /= np.linalg.norm(Q[i])
    return Q


def biorthonormalize(c_phi, c_chi):
    """(phi, chi) per k: phi orthonormal, chi biorthonormal to phi, chi spanning the input chi."""
    c_phi = np.asarray(c_phi, dtype=np.complex128)
    c_chi = np.asarray(c_chi, dtype=np.complex128)
    out_phi = np.empty_like(c_phi)
    out_chi = np.empty_like(c_chi)
    for k in range(c_phi.shape[0]):
        phi = gram_schmidt(c_phi[k])
        M = np.conj(phi) @ c_chi[k].T            # M[i, j] = <phi_i|chi'_j>
        out_phi[k] = phi
        out_chi[k] = np.linalg.inv(M).T @ c_chi[k]   # chi_j = sum_i (M^-1)[i, j] chi'_i
    return out_phi, out_chi
