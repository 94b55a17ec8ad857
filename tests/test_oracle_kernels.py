"""Pins of the oracle's kernel transforms against quadrature and limits (Sec. 2.6.3, App. B)."""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import kernels as KN

PARAMS = [(1.63886, 1.81045), (1.63886, 1.28018), (4.61880, 3.03934), (0.7, 0.4)]


def _radial_ft(f, p, R, tail_c3=0.0):
    """int d^3r f(r) e^{-ip.r} = (4 pi / p) int_0^inf r f(r) sin(p r) dr.

    The range [0, R] is integrated piecewise (one panel per half period); beyond
    R the integrand is tail_c3 sin(pr)/r^3, integrated in closed form with Si.
    """
    edges = np.unique(np.concatenate([[0.0], np.arange(1, int(p * R / np.pi) + 1) * np.pi / p, [R]]))
    head = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        v, _ = integrate.quad(lambda r: r * f(r) * np.sin(p * r), a, b, epsabs=1e-300, epsrel=1e-13, limit=200)
        head += v
    X = p * R
    si, _ = special.sici(X)
    i3 = np.sin(X) / (2 * X * X) + np.cos(X) / (2 * X) - 0.5 * (0.5 * np.pi - si)
    return 4.0 * np.pi / p * (head + tail_c3 * p * p * i3)


@pytest.mark.parametrize("A,C", PARAMS)
def test_grad_u_squared_matches_radial_quadrature(A, C):
    def gu2(r):
        # (grad u)^2 = (A^2/r^2) (e^{-r/C}/C + (e^{-r/C} - 1)/r)^2  (Appendix B)
        if r < 1e-6:
            return (A / (2 * C * C)) ** 2
        return (A / r) ** 2 * (np.exp(-r / C) / C + np.expm1(-r / C) / r) ** 2

    for g in [0.05, 0.5, 0.999, 1.001, 3.0, 5.999, 6.001, 15.0, 40.0]:
        p = g / C
        ref = _radial_ft(gu2, p, R=45.0 * C, tail_c3=A * A)
        val = KN.gradu_sq(np.array([p]), A, C)[0]
        assert abs(val - ref) <= 1e-9 * abs(ref), (g, val, ref)


@pytest.mark.parametrize("A,C", PARAMS)
def test_laplacian_u_matches_quadrature_and_u_tilde(A, C):
    # lap u = u'' + 2u'/r for u = A(1 - e^{-r/C})/r equals -A e^{-r/C}/(C^2 r) away from r = 0
    # (the delta functions of the two 1/r parts cancel).
    def lap(r):
        return -A * np.exp(-r / C) / (C * C * r)

    for p in [0.1, 0.7, 2.0, 9.0]:
        ref = _radial_ft(lap, p, R=45.0 * C)
        assert abs(KN.lap_u(p * p, A, C) - ref) <= 1e-10 * abs(ref)
        assert abs(-p * p * KN.u_tilde(p * p, A, C) - KN.lap_u(p * p, A, C)) <= 1e-14 * abs(ref)


@pytest.mark.parametrize("A,C", PARAMS)
def test_limits_and_asymptotes(A, C):
    # (grad u)^2 at p -> 0 is 2 pi A^2 / C, approached linearly with slope -(pi/4)(4 pi A^2/C) C
    p = np.array([1e-7])
    assert abs(KN.gradu_sq(p, A, C)[0] - 2 * np.pi * A * A / C) < 1e-12 * A * A / C + 4 * np.pi * A * A * 1e-7
    assert KN.gradu_sq(np.array([0.0]), A, C)[0] == 2 * np.pi * A * A / C
    # large p: 8 pi A^2 / (3 C^5 p^4)
    for g in [200.0, 1e3]:
        p = g / C
        asym = 8 * np.pi * A * A / (3 * C ** 5 * p ** 4)
        assert abs(KN.gradu_sq(np.array([p]), A, C)[0] / asym - 1.0) < 20.0 / g ** 2
    # lap u at 0 and u_short
    assert abs(KN.lap_u(0.0, A, C) + 4 * np.pi * A) < 1e-13 * A
    q2 = 1e-6
    assert abs((KN.u_tilde(q2, A, C) - 4 * np.pi * A / q2) - KN.u_short(A, C)) < 1e-4 * abs(KN.u_short(A, C))


def test_grad_u_squared_branches_are_continuous():
    A, C = 1.3, 0.9
    for g0 in (1.0, 6.0):
        gs = np.array([g0 * (1 - 1e-12), g0 * (1 + 1e-12)])
        v = KN.gradu_sq(gs / C, A, C)
        assert abs(v[0] - v[1]) < 1e-11 * abs(v[0])


def test_V2a_and_dagger():
    A, C = 1.63886, 1.81045
    for p2 in [0.01, 0.4, 3.0]:
        V = KN.V2a(p2, A, C)
        Vd = KN.V2a(p2, A, C, adjoint=True)
        assert abs((Vd - V) - 2 * p2 * KN.u_tilde(p2, A, C)) < 1e-12 * abs(V)
        assert abs(V - (4 * np.pi / p2 + KN.lap_u(p2, A, C) - KN.gradu_sq(np.array([np.sqrt(p2)]), A, C)[0])) < 1e-12 * abs(V)
    assert KN.V2a_jastrow_zero(A, C) == pytest.approx(-4 * np.pi * A - 2 * np.pi * A * A / C, rel=1e-15)
