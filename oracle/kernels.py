"""Fourier transforms of the Jastrow-derived interactions (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Jastrow function u(r) = A/r (1 - exp(-r/C)) (Eq. Jastrow).  Non-periodic Fourier
transforms (Sec. 2.2 convention, g~(G) = int dr g(r) e^{-iG.r}):

* u~(p)          = 4 pi A (1/p^2 - 1/(p^2 + C^-2))      (Sec. 2.6.3)
* (lap u)~(p)    = -p^2 u~(p) = -4 pi A C^-2/(p^2 + C^-2)
* ((grad u)^2)~  = (4 pi A^2/(C g)) B(g), g = C p, with
  B(g) = -(pi/4) g^2 - (1 + g^2/2) atan(g/2) + (1 + g^2) atan(g)   (Eq. fourier_transform_nabla2u, App. B)
* V_2a(p)        = 4 pi/p^2 + (lap u)~ - ((grad u)^2)~   (Sec. 2.6.3: 1/r + (1/2)[lap1 u + lap2 u
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

    The Coulomb 4 pi/p^2 part is the only divergent piece (Sec. 2.6.3, after
    Eq. divcorr_2ax_scf); it is dropped at p = 0 and replaced by the divergence
    correction.  The same value is used for V_2a^dagger: on the grid the
    grad u . grad terms vanish at p = 0 (their kernel i p u~ is set to zero there), so the
    integration by parts that flips the sign of lap u does not apply at that point, and the
    adjoint of the discrete right operator keeps -4 pi A.
    """
    return -FOUR_PI * A - 2.0 * np.pi * A * A / C


# ---------------------------------------------------------------------------
# Derivatives with respect to the Jastrow parameters A and C, for dE/dA and
# dE/dC.  They follow by differentiating the closed forms above; with
# g = C p and D(g) = g B'(g) - 2 B(g):
#   du~/dA        = 4 pi C^-2 / (p^2 (p^2 + C^-2))
#   du~/dC        = -8 pi A / (C^3 (p^2 + C^-2)^2)
#   d(lap u)~/dA  = -4 pi C^-2 / (p^2 + C^-2)
#   d(lap u)~/dC  = 8 pi A p^2 / (C^3 (p^2 + C^-2)^2)
#   d((grad u)^2)~/dA = (8 pi A / (C g)) B(g)            (limit 4 pi A / C at p = 0)
#   d((grad u)^2)~/dC = (4 pi A^2 / (C^3 p)) D(g)        (limit -2 pi A^2 / C^2 at p = 0)
# B'(g) = 2/(4 + g^2) + g (2 atan g - atan(g/2) - pi/2); for g > 1 the bracket is
# atan(2/g) - 2 atan(1/g) (pi terms cancelled as for B), and for g > 6 the series of
# B gives D(g) = -sum_k (2k + 3) c_k g^-(2k+1).
# Parity pins: tests/test_oracle_gradient.py compares each with central
# differences of the value functions on all three branches of B.

def du_dA(p2, C):
    c2 = 1.0 / (C * C)
    return FOUR_PI * c2 / (p2 * (p2 + c2))


def du_dC(p2, A, C):
    c2 = 1.0 / (C * C)
    return -2.0 * FOUR_PI * A / (C ** 3 * (p2 + c2) ** 2)


def dlap_dA(p2, C):
    c2 = 1.0 / (C * C)
    return -FOUR_PI * c2 / (p2 + c2)


def dlap_dC(p2, A, C):
    c2 = 1.0 / (C * C)
    return 2.0 * FOUR_PI * A * p2 / (C ** 3 * (p2 + c2) ** 2)


def _D_direct(g):
    dB = 2.0 / (4.0 + g * g) + g * (2.0 * np.arctan(g) - np.arctan(0.5 * g) - 0.5 * np.pi)
    return g * dB - 2.0 * _B_direct(g)


def _D_reflect(g):
    dB = 2.0 / (4.0 + g * g) + g * (np.arctan(2.0 / g) - 2.0 * np.arctan(1.0 / g))
    return g * dB - 2.0 * _B_reflect(g)


def _D_series(g):
    out = np.zeros_like(g)
    inv2 = 1.0 / (g * g)
    term_pow = inv2 / g
    for k in range(1, 60):
        ck = (-1) ** k * ((2.0 ** (2 * k + 1) - 1.0) / (2 * k + 1) - (2.0 ** (2 * k + 2) - 1.0) / (2 * k + 3))
        out = out - (2 * k + 3) * ck * term_pow
        term_pow = term_pow * inv2
    return out


def D_of_g(g):
    """D(g) = g B'(g) - 2 B(g), on the same three branches as B_of_g."""
    g = np.asarray(g, dtype=np.float64)
    out = np.empty_like(g)
    s = g <= 1.0
    m = (g > 1.0) & (g <= 6.0)
    l = g > 6.0
    out[s] = _D_direct(g[s])
    out[m] = _D_reflect(g[m])
    out[l] = _D_series(g[l])
    return out


def dgradu_sq_dA(p, A, C):
    p = np.asarray(p, dtype=np.float64)
    g = C * p
    out = np.empty_like(g)
    z = g == 0.0
    out[z] = FOUR_PI * A / C
    out[~z] = 2.0 * FOUR_PI * A / (C * g[~z]) * B_of_g(g[~z])
    return out


def dgradu_sq_dC(p, A, C):
    p = np.asarray(p, dtype=np.float64)
    g = C * p
    out = np.empty_like(g)
    z = g == 0.0
    out[z] = -2.0 * np.pi * A * A / (C * C)
    out[~z] = FOUR_PI * A * A / (C ** 3 * p[~z]) * D_of_g(g[~z])
    return out


class JastrowKernels:
    """Jastrow-dependent kernel data of the operator, per spin channel s (0 parallel, 1 antiparallel).

    With ``deriv=None`` the methods return the kernels themselves; with
    ``deriv=("A", s0)`` or ``("C", s0)`` they return the derivatives with respect
    to that parameter (zero for the other channel, and zero for the Coulomb part).
    All functions are without the 1/Omega of the operator.

      coulomb(p2)               4 pi / p^2
      coulomb_zero(Nk, Gamma0)  replacement of the Coulomb part at p = 0 (Eq. divcorr_2ax_scf)
      u(p2, s), lap(p2, s), gsq(p, s), V2a(p2, s, adjoint)
      v0(s)                     finite Jastrow part of V_2a at p = 0, (lap u)~(0) - ((grad u)^2)~(0)
      amp(s)                    A_s (the 4 pi A_s / N_k of the 3a2 and 3b6 corrections)
      corr(s, Gamma0, x, Nk)    (4 pi A_s)^2 Gamma0 + x 4 pi A_s u_short,s / N_k
    """

    def __init__(self, A, C, deriv=None):
        self.A = np.asarray(A, dtype=np.float64)
        self.C = np.asarray(C, dtype=np.float64)
        self.deriv = deriv

    def _on(self, s):
        return self.deriv is None or self.deriv[1] == s

    def _wrt(self):
        return None if self.deriv is None else self.deriv[0]

    def coulomb(self, p2):
        return FOUR_PI / p2 if self.deriv is None else np.zeros_like(p2)

    def coulomb_zero(self, Nk, Gamma0):
        return FOUR_PI * Nk * Gamma0 if self.deriv is None else 0.0

    def u(self, p2, s):
        A, C = self.A[s], self.C[s]
        if not self._on(s):
            return np.zeros_like(p2)
        w = self._wrt()
        return u_tilde(p2, A, C) if w is None else (du_dA(p2, C) if w == "A" else du_dC(p2, A, C))

    def lap(self, p2, s):
        A, C = self.A[s], self.C[s]
        if not self._on(s):
            return np.zeros_like(p2)
        w = self._wrt()
        return lap_u(p2, A, C) if w is None else (dlap_dA(p2, C) if w == "A" else dlap_dC(p2, A, C))

    def gsq(self, p, s):
        A, C = self.A[s], self.C[s]
        if not self._on(s):
            return np.zeros_like(np.asarray(p, dtype=np.float64))
        w = self._wrt()
        return gradu_sq(p, A, C) if w is None else (dgradu_sq_dA(p, A, C) if w == "A" else dgradu_sq_dC(p, A, C))

    def V2a(self, p2, s, adjoint=False):
        sgn = -1.0 if adjoint else 1.0
        return self.coulomb(p2) + sgn * self.lap(p2, s) - self.gsq(np.sqrt(p2), s)

    def v0(self, s):
        A, C = self.A[s], self.C[s]
        if not self._on(s):
            return 0.0
        w = self._wrt()
        if w is None:
            return V2a_jastrow_zero(A, C)
        return -FOUR_PI - FOUR_PI * A / C if w == "A" else 2.0 * np.pi * A * A / (C * C)

    def amp(self, s):
        if not self._on(s):
            return 0.0
        w = self._wrt()
        return self.A[s] if w is None else (1.0 if w == "A" else 0.0)

    def corr(self, s, Gamma0, x, Nk):
        A, C = self.A[s], self.C[s]
        if not self._on(s):
            return 0.0
        w = self._wrt()
        a2 = (FOUR_PI * A) ** 2
        if w is None:
            return a2 * Gamma0 + x * FOUR_PI * A * u_short(A, C) / Nk
        if w == "A":
            return 2.0 * FOUR_PI ** 2 * A * (Gamma0 - x * C * C / Nk)
        return a2 * (-2.0 * x * C / Nk)


class DisplacedKernels:
    """base + t * direction for every kernel datum (base and direction are JastrowKernels)."""

    def __init__(self, base, direction, t):
        self.b, self.d, self.t = base, direction, float(t)

    def __getattr__(self, name):
        fb, fd, t = getattr(self.b, name), getattr(self.d, name), self.t
        return lambda *a, **kw: fb(*a, **kw) + t * fd(*a, **kw)
