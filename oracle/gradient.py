"""Gradient of the TC pseudo-energy (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

E is the pseudo-energy of ``operator.energy_terms`` (Eqs. EtotTC / EtotBiTC):
E = (2/N_k) Re sum_j f_j [<chi_j|T|phi_j> + (1/2) <chi_j|g2_j> + (1/3) <chi_j|g3_j>],
with f_j = 0 for every band j >= nocc (the bands that act as partners are the
bands that carry weight in E).

Gradient convention: for a real function of complex coefficients c the
gradient is g = dE/dRe(c) + i dE/dIm(c), so that dE = Re sum conj(g) dc (the
convention of PyTorch for real-valued functions of complex tensors).

Orbitals.  E depends on the ket coefficients phi and on the conjugated bra
coefficients chi^*.  The two- and three-body operators are the derivatives of
the two- and three-body parts of E (an identity of the single-determinant
energy, pinned exactly below), so
    g_chi = (2/N_k) f (T phi + h phi)        (right operator output),
    g_phi = (2/N_k) f (T chi + h^dagger chi) (left operator output).
With the SCF-mesh divergence corrections included this still holds: the 2ax
correction is a symmetric quadratic form of the overlaps, and the 3a2 and 3b6
correction energies are one cubic form of overlaps and pair spectra whose
derivatives through its three pair factors are exactly the 3a2 correction
(through the density) and the 3b6 correction (through the two other pairs).

Jastrow parameters.  E depends on (A_s, C_s), s in {pp, ap}, only through the
kernel data: the tables u~_s, (lap u)~_s, ((grad u)^2)~_s, the p = 0 value of
V_2a and the coefficients (4 pi A_s)^2 Gamma0 + x 4 pi A_s u_short,s / N_k and
4 pi A_s / N_k of the corrections.  Every term of the operator is linear in one
kernel datum or a product of two, so E is a polynomial of degree 2 in the
kernel data K.  Hence along the derivative direction dK = dK/dtheta,
    dE/dtheta = [E(K + t dK) - E(K - t dK)] / (2 t)
holds for any t without truncation error.  dK comes from
``kernels.JastrowKernels(deriv=...)`` (closed-form derivatives of the
transforms of Sec. 2.6.3 and Appendix B).

Parity pins (tests/test_oracle_gradient.py): the orbital gradient against an
exact 4-point stencil of E along random directions, corrections on and off,
and with occupations that differ between k-points;
dE/dA_s against the exact 3-point difference of E (E is quadratic in A_s at
fixed C); dE/dC_s against Richardson-extrapolated central differences of E;
the degree-2 claim along dK; each kernel derivative against central
differences of the kernel itself.
"""
import numpy as np

from . import kernels as KN
from . import operator as OP


def orbital_gradient(S, c_phi, c_chi, occ, backend=None):
    """(g_phi, g_chi): gradients of E with respect to the right and left coefficients."""
    occ = np.asarray(occ, dtype=np.float64).reshape(S.Nk, S.nbands)
    if np.any(occ[:, S.nocc:] != 0.0):
        raise ValueError("the energy gradient needs f = 0 for bands >= nocc")
    out_r, out_l = OP.tc_apply(S, c_phi, c_chi, occ, backend=backend)
    w = (2.0 / S.Nk) * occ[:, :, None]
    g_phi = w * (OP.kinetic_coeffs(S, np.asarray(c_chi, dtype=np.complex128)) + out_l)
    g_chi = w * (OP.kinetic_coeffs(S, np.asarray(c_phi, dtype=np.complex128)) + out_r)
    return g_phi, g_chi


def displacement(theta):
    """Step t of the symmetric difference along dK (any t is exact; this one keeps rounding small)."""
    return 0.5 * max(abs(theta), 0.1)


def param_gradient(S, c_phi, c_chi, occ, backend=None):
    """{"A": [dE/dA_pp, dE/dA_ap], "C": [dE/dC_pp, dE/dC_ap]} at fixed orbitals."""
    base = KN.JastrowKernels(S.A, S.C)
    out = {"A": [0.0, 0.0], "C": [0.0, 0.0]}
    for name, vals in (("A", S.A), ("C", S.C)):
        for s in range(2):
            d = KN.JastrowKernels(S.A, S.C, deriv=(name, s))
            t = displacement(vals[s])
            ep = OP.energy_terms(S, c_phi, c_chi, occ, backend=backend,
                                 kset=KN.DisplacedKernels(base, d, +t))["total"]
            em = OP.energy_terms(S, c_phi, c_chi, occ, backend=backend,
                                 kset=KN.DisplacedKernels(base, d, -t))["total"]
            out[name][s] = (ep - em) / (2.0 * t)
    return out
