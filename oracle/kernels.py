"""Fourier transforms of the Jastrow-derived interactions (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Jastrow function u(r) = A/r (1 - exp(-r/C)) (Eq. Jastrow).  Non-periodic Fourier
transforms (Sec. 2.2 convention, g~(G) = int dr g(r) e^{-iG.r}):

* u~(p)          = 4 pi A (1/p^2 - 1/(p^2 + C^-2))      (Sec. 2.7.3)
* (lap u)~(p)    = -p^2 u~(p) = -4 pi A C^-2/(p^2 + C^-2)
* ((grad u)^2)~  = (4 pi A^2/(C g)) B(g), g = C p, with
  B(g) = -(pi/4) g^2 - (1 + g^2/2) atan(g/2) + (1 + g^2) atan(g)   (Eq. fourier_transform_nabla2u, App. B)
* V_2a(p)        = 4 pi/p^2 + (lap u)~ - ((grad u)^2)~   (Sec. 2.7.3: 1/r + (1/2)[lap1 u + lap2 u
                   - (grad1 u)^2 - (grad2 u)^2], both Laplacians and both squared
                   gradients being the same function of r1 - r2)
* V_2a^dagger(p) = 4 pi/p^2 - (lap u)~ - ((grad u)^2)~  (the 1/r + ... part of v_2body^dagger:
                   the adjoint of grad u . grad is -lap u - grad u . grad)

Numerics of B(g): the printed form cancels badly for large g.  For g > 1 the
identity atan(x) = pi/2 - atan(1/x) removes the pi terms exactly,
B(g) = (1 + g^2/2) atan(2/g) - (1 + g^2) atan(1/g); for g > 6 the Taylor
series of atan in 1/g gives B(g) = sum_k c_k g^-(2k+1) with
c_k = (-1)^k [(2^(2k+1) - 1)/(2k+1) - (2^(2k+2) - 1)/(2k+3)] (c_0 = 0, c_1 = 2/3,
c_2 = -14/5).  Limits: u~ ~ 4 pi A/p^2 + u_short with u_short = -4 pi A C^2
(Eq. u_short); (lap u)~(0) = -4 pi A; ((grad u)^2)~(0) = 2 pi A^2 / C.

Parity pins: ``tests/test_oracle_kernels.py`` checks every transform against
radial quadrature of its real-space definition, the limits above, and the
large-p asymptote 8 pi A^2 / (3 C^5 p^4) of ((grad u)^2)~.
"""
import numpy as np

FOUR_PI = 4.0 * np.pi


def u_tilde(p2, A, C):
    """u~ at p^2 > 0, in the cancellation-free form 4 pi A C^-2 / (p^2 (p^2 + C^-2))."""
    c2 = 1.0 / (C * C)
    return FOUR_PI * A * c2 / (p2 * (p2 + c2))


def lap_u(p2, A, C):
    c2 = 1.0 / (C * C)
    return -FOUR_PI * A * c2 / (p2 + c2)


def _B_direct(g):
    return -0.25 * np.pi * g * g - (1.0 + 0.5 * g * g) * np.arctan(0.5 * g) + (1.0 + g * g) * np.arctan(g)


def _B_reflect(g):
    return (1.0 + 0.5 * g * g) * np.arctan(2.0 / g) - (1.0 + g * g) * np.arctan(1.0 / g)


def _B_series(g):
    out = np.zeros_like(g)
    inv = 1.0 / g
    inv2 = inv * inv
    term_pow = inv * inv2          # g^-3 for k = 1
    for k in range(1, 60):
        ck = (-1) ** k * ((2.0 ** (2 * k + 1) - 1.0) / (2 * k + 1) - (2.0 ** (2 * k + 2) - 1.0) / (2 * k + 3))
        out = out + ck * term_pow
        term_pow = term_pow * inv2
    return out


def B_of_g(g):
    """B(g) of Appendix B, evaluated stably (see module docstring)."""
    g = np.asarray(g, dtype=np.float64)
    out = np.empty_like(g)
    s = g <= 1.0
    m = (g > 1.0) & (g <= 6.0)
    l = g > 6.0
    out[s] = _B_direct(g[s])
    out[m] = _B_reflect(g[m])
    out[l] = _B_series(g[l])
    return out


def gradu_sq(p, A, C):
    """((grad u)^2)~ at |p| = p (p >= 0); the p = 0 value is the limit 2 pi A^2 / C."""
    p = np.asarray(p, dtype=np.float64)
    g = C * p
    out = np.empty_like(g)
    z = g == 0.0
    out[z] = 2.0 * np.pi * A * A / C
    nz = ~z
    out[nz] = FOUR_PI * A * A / (C * g[nz]) * B_of_g(g[nz])
    return out


def u_short(A, C):
    """lim_{p->0} [u~(p) - 4 pi A/p^2] (Eq. u_short)."""
    return -FOUR_PI * A * C * C


def V2a(p2, A, C, adjoint=False):
    """V_2a (or V_2a^dagger) at p^2 > 0."""
    p = np.sqrt(p2)
    lap = lap_u(p2, A, C)
    s = -1.0 if adjoint else 1.0
    return FOUR_PI / p2 + s * lap - gradu_sq(p, A, C)


def V2a_jastrow_zero(A, C):
    """Finite Jastrow part of V_2a at p = 0: (lap u)~(0) - ((grad u)^2)~(0).

    The Coulomb 4 pi/p^2 part is the only divergent piece (Sec. 2.7.3, after
    Eq. divcorr_2ax_scf); it is dropped at p = 0 and replaced by the divergence
    correction.  The same value is used for V_2a^dagger: on the grid the
    grad u . grad terms vanish at p = 0 (their kernel i p u~ is set to zero there), so the
    integration by parts that flips the sign of lap u does not apply at that point, and the
    adjoint of the discrete right operator keeps -4 pi A.
    """
    return -FOUR_PI * A - 2.0 * np.pi * A * A / C
