"""One block-Davidson step for the non-Hermitian TC one-body operator (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.4 treats the SCF equation as the eigenvalue problem of the non-Hermitian
operator h built from the current orbitals and solves it per k-point by block
Davidson.  This module takes one step with p_max = 1, i.e. a subspace of two
blocks (the default block count of the paper's input table):

1. the trial vectors v_i (i < m) are the current right orbitals, orthonormal
   per k; their estimates are eps_i = <v_i|h|v_i>, which for Gram-Schmidt
   orthonormalised eigenvectors equals the eigenvalue (Appendix A);
2. the new block is w_i = P (h - eps_i) v_i, with Payne's preconditioner
   P(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4) acting
   per plane wave, x(G) = |k+G|^2/2 divided by the kinetic energy
   sum_G' |k+G'|^2/2 |v_i(G')|^2 of the trial vector;
3. each w_i, in order, is orthogonalised against all vectors kept so far and
   normalised; one whose norm is below 1e-8 at that point is left out, so the
   subspace dimension d can be smaller than 2m;
4. the subspace matrix is M_ab = <b_a|h|b_b> over the orthonormal basis
   b = (v_0 .. v_{m-1}, kept w);
5. M's right eigenvectors y and left eigenvectors z, normalised so that
   z^H y = 1 (z = rows of y^-1, conjugated), are ordered by the real part of
   the eigenvalue; the lowest m give phi_i = sum_a y_ai b_a and
   chi_i = sum_a z_ai b_a -- left and right solutions expanded in the same
   trial vectors, as BITC needs (Sec. 2.4);
6. phi is orthonormalised by Gram-Schmidt and chi made biorthonormal to it
   (``biortho.biorthonormalize``): the trial vectors of the next step.

h here is the kinetic term plus the two- and three-body TC operator of
``operator.py`` (the cells have no pseudopotential).  During the step the
partners (the first nocc bands with their occupations) stay fixed; h acts on
a vector placed in an unoccupied band of a set whose first nocc bands are the
partners.

``davidson_dense`` takes the same steps with an explicit matrix for h; it is
what the pins use to compare against a brute-force eigen-decomposition.

Parity pins (tests/test_oracle_davidson.py): with 2m >= the vector length
the step is exact and returns the lowest m eigenpairs of the full matrix;
trial vectors that span an invariant subspace give no new direction and
return their own eigenvalues; Appendix A (the Gram-Schmidt of eigenvectors
keeps the eigenvalues on the diagonal and zeros below it); z^H y = I and
the eigen-equations; plane waves of the homogeneous electron gas are exact
eigenvectors of the TC operator, with the closed-form eigenvalues; the
Payne factor's values and limits, its argument for one- and two-wave trial
vectors, and the 1e-8 norm cut on both sides.
"""
import copy

import numpy as np

from . import biortho as BO
from . import operator as OP

NORM_CUT = 1e-8


def payne(x):
    """Payne preconditioner P(x) (Sec. 2.4)."""
    x = np.asarray(x, dtype=np.float64)
    num = 27.0 + 18.0 * x + 12.0 * x * x + 8.0 * x ** 3
    return num / (num + 16.0 * x ** 4)


def payne_vector(t, ekin):
    """P(x(G)) over a sphere: t = |k+G|^2/2 per plane wave, ekin = <v|T|v> of the trial vector.

    A trial vector with zero kinetic energy (the k+G = 0 plane wave alone) takes the
    ekin -> 0 limit: P = 1 where t = 0 and P = 0 elsewhere.
    """
    if ekin > 0.0:
        return payne(t / ekin)
    return (t == 0.0).astype(np.float64)


def eig_sorted(M):
    """(lambda, y, z) of a square matrix: M y = y diag(lambda), z^H M = diag(lambda) z^H, z^H y = I.

    Eigenpairs in ascending order of the real part of lambda.
    """
    lam, y = np.linalg.eig(M)
    order = np.argsort(lam.real, kind="stable")
    lam, y = lam[order], y[:, order]
    z = np.linalg.inv(y).conj().T
    return lam, y, z


def new_directions(v, hv, t):
    """Steps 1-3 for one k: the kept new vectors (list, in order) and their indices.

    v, hv: (m, n) trial vectors (orthonormal rows) and h applied to them;
    t: (n,) kinetic energy |k+G|^2/2 of each plane wave (zero where padded).
    """
    m = v.shape[0]
    basis = [v[i] for i in range(m)]
    kept, idx = [], []
    for i in range(m):
        eps = np.vdot(v[i], hv[i])
        ekin = float(np.real(np.vdot(v[i], t * v[i])))
        u = payne_vector(t, ekin) * (hv[i] - eps * v[i])
        for b in basis:
            u = u - np.vdot(b, u) * b
        nrm = np.linalg.norm(u)
        if nrm < NORM_CUT:
            continue
        u = u / nrm
        basis.append(u)
        kept.append(u)
        idx.append(i)
    return kept, idx


def subspace_solve(B, HB, m):
    """Steps 4-5 for one k: (lambda[:m], phi (m, n), chi (m, n)) from basis rows B and h B."""
    M = np.conj(B) @ HB.T                       # M[a, b] = <b_a|h|b_b>
    lam, y, z = eig_sorted(M)
    return lam[:m], y[:, :m].T @ B, z[:, :m].T @ B


def davidson_dense(H, v, t):
    """One step with an explicit matrix h = H (n, n) on the rows of v (m, n).

    Returns (lambda (m,), phi (m, n), chi (m, n), d).
    """
    v = np.asarray(v, dtype=np.complex128)
    m = v.shape[0]
    hv = v @ H.T
    kept, _ = new_directions(v, hv, t)
    B = np.array([*v, *kept])
    lam, phi, chi = subspace_solve(B, B @ H.T, m)
    phi, chi = BO.biorthonormalize(phi[None], chi[None])
    return lam, phi[0], chi[0], B.shape[0]


def kinetic_diag(S, k):
    """(npw_max,) |k+G|^2/2 over the sphere of k-point k, zero padded."""
    t = np.zeros(S.npw_max)
    kg = S.kpG(k)
    t[: S.npw[k]] = 0.5 * np.einsum("ij,ij->i", kg, kg)
    return t


def h_apply(S, c_phi, c_chi, occ, vecs):
    """(T + h2 + h3) vecs[k, i] for every k, with the first nocc bands of (c_phi, c_chi, occ) as partners."""
    no = S.nocc
    Nk, nv = vecs.shape[0], vecs.shape[1]
    S2 = copy.copy(S)
    S2.nbands = no + nv
    phi = np.concatenate([c_phi[:, :no], vecs], axis=1)
    chi = np.concatenate([c_chi[:, :no], vecs], axis=1)
    occ2 = np.concatenate([np.asarray(occ, dtype=np.float64).reshape(Nk, -1)[:, :no], np.zeros((Nk, nv))], axis=1)
    out = OP.total(OP.apply_operator(S2, phi, chi, occ2, left=False))
    return (OP.kinetic_coeffs(S2, phi) + out)[:, no:]


def davidson_step(S, c_phi, c_chi, occ):
    """One step for every band of every k-point.

    S: Setup with nbands = m, nocc partners; c_phi (Nk, m, npw_max) orthonormal per k,
    c_chi biorthonormal to it; occ (Nk, m).
    Returns (phi, chi, lambda (Nk, m) complex, d (Nk,) subspace dimensions).
    """
    c_phi = np.asarray(c_phi, dtype=np.complex128)
    c_chi = np.asarray(c_chi, dtype=np.complex128)
    Nk, m = c_phi.shape[0], c_phi.shape[1]
    v = c_phi
    hv = h_apply(S, c_phi, c_chi, occ, v)
    w = np.zeros_like(v)
    nkept = np.zeros(Nk, dtype=int)
    for k in range(Nk):
        kept, _ = new_directions(v[k], hv[k], kinetic_diag(S, k))
        nkept[k] = len(kept)
        for a, u in enumerate(kept):
            w[k, a] = u
    hw = h_apply(S, c_phi, c_chi, occ, w)
    phi = np.zeros_like(v)
    chi = np.zeros_like(v)
    lam = np.zeros((Nk, m), dtype=np.complex128)
    for k in range(Nk):
        B = np.concatenate([v[k], w[k, : nkept[k]]])
        HB = np.concatenate([hv[k], hw[k, : nkept[k]]])
        lam[k], phi[k], chi[k] = subspace_solve(B, HB, m)
    phi, chi = BO.biorthonormalize(phi, chi)
    return phi, chi, lam, m + nkept
