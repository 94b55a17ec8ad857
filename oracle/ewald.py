"""Ewald sum of the Madelung potential of a point-charge lattice (oracle pin).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Potential at a lattice site of unit point charges on the lattice spanned by
the rows of ``S`` in a uniform neutralising background (textbook Ewald split,
screening parameter eta):

  v_M = sum'_R erfc(sqrt(eta) R)/R + (4 pi/V) sum'_G exp(-G^2/(4 eta))/G^2
        - pi/(eta V) - 2 sqrt(eta/pi).

Used only to pin the divergence-correction constant: for k on the SCF mesh,
4 pi Gamma0 / Omega equals -v_M of the Born-von Karman supercell (the
auxiliary-function sum of Eq. correction2 is the reciprocal half of this Ewald
sum with alpha = 1/(4 eta), the real-space half being negligible when
sqrt(alpha) <= L_min/12).

``phased_sum`` is the same split of S(k) = sum_{R != 0} cos(k.R)/R for a wave
vector k off the reciprocal lattice of S (no K = 0 term and no background):

  S(k) = sum_{R != 0} cos(k.R) erfc(sqrt(eta) R)/R
         + (4 pi/V) sum_K exp(-|k - K|^2/(4 eta))/|k - K|^2 - 2 sqrt(eta/pi),

which pins the band-point constant: 4 pi Gamma_b(k)/Omega = -S(k) for the
Born-von Karman supercell.
"""
import math

import numpy as np
from scipy.special import erfc


def madelung(S, eta=None, tol=1e-17):
    S = np.asarray(S, dtype=np.float64)
    V = abs(np.linalg.det(S))
    B = 2.0 * np.pi * np.linalg.inv(S).T
    Lmin = min(np.linalg.norm(S, axis=1))
    if eta is None:
        eta = (2.2 / Lmin) ** 2
    rcut = np.sqrt(-np.log(tol)) / np.sqrt(eta) + Lmin
    gcut = 2.0 * np.sqrt(eta) * np.sqrt(-np.log(tol))
    nr = [int(np.ceil(rcut * np.linalg.norm(B[i]) / (2 * np.pi))) + 1 for i in range(3)]
    ng = [int(np.ceil(gcut * np.linalg.norm(S[i]) / (2 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-x, x + 1) for x in nr]
    l = np.stack(np.meshgrid(*r, indexing="ij"), -1).reshape(-1, 3)
    R = np.linalg.norm(l @ S, axis=1)
    R = R[R > 0]
    real = np.sum(np.sort(erfc(np.sqrt(eta) * R) / R))
    g = [np.arange(-x, x + 1) for x in ng]
    l = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
    G2 = np.einsum("ij,ij->i", l @ B, l @ B)
    G2 = G2[G2 > 0]
    recip = 4.0 * np.pi / V * np.sum(np.sort(np.exp(-G2 / (4.0 * eta)) / G2))
    return real + recip - np.pi / (eta * V) - 2.0 * np.sqrt(eta / np.pi)


def phased_sum(S, k, eta=None, tol=1e-17):
    """S(k) = sum_{R != 0} cos(k.R)/R over the lattice rows of S (Ewald split), k off its reciprocal lattice."""
    S = np.asarray(S, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    V = abs(np.linalg.det(S))
    B = 2.0 * np.pi * np.linalg.inv(S).T
    Lmin = min(np.linalg.norm(S, axis=1))
    if eta is None:
        eta = (2.2 / Lmin) ** 2
    rcut = np.sqrt(-np.log(tol)) / np.sqrt(eta) + Lmin
    gcut = 2.0 * np.sqrt(eta) * np.sqrt(-np.log(tol)) + np.linalg.norm(k)
    nr = [int(np.ceil(rcut * np.linalg.norm(B[i]) / (2 * np.pi))) + 1 for i in range(3)]
    ng = [int(np.ceil(gcut * np.linalg.norm(S[i]) / (2 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-x, x + 1) for x in nr]
    Rv = np.stack(np.meshgrid(*r, indexing="ij"), -1).reshape(-1, 3) @ S
    R = np.linalg.norm(Rv, axis=1)
    keep = R > 0
    real = math.fsum(np.cos(Rv[keep] @ k) * erfc(np.sqrt(eta) * R[keep]) / R[keep])
    g = [np.arange(-x, x + 1) for x in ng]
    P = k[None, :] - np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3) @ B
    P2 = np.einsum("ij,ij->i", P, P)
    if np.any(P2 == 0.0):
        raise ValueError("k lies on the reciprocal lattice")
    recip = 4.0 * np.pi / V * math.fsum(np.exp(-P2 / (4.0 * eta)) / P2)
    return real + recip - 2.0 * np.sqrt(eta / np.pi)
