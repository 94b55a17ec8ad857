"""Pins of the oracle's energy gradient (oracle/gradient.py): orbitals, A and C.

Every pin compares with finite differences of the oracle's energy itself, which
uses only the kernel values, never the derivative kernels.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import gradient as GR
from oracle import kernels as KN
from oracle import operator as OP
from paper_2302_07420_gb300 import synth

PARAMS = [(1.63886, 1.81045), (1.63886, 1.28018), (4.61880, 3.03934), (0.7, 0.4)]


def tiny(seed=0, div=1, ushort_factor=1.0, fill=(1.0, 0.6), A=None, C=None):
    p = synth.tiny_params(seed, kmesh=(1, 1, 2), fft=(9, 9, 11), ecut=1.6, nbands=3, nocc=2, scale=5.0)
    kw = dict(div_correction=div, ushort_factor=ushort_factor)
    if A is not None:
        kw["A"] = A
    if C is not None:
        kw["C"] = C
    S = make_setup(p, **kw)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 90 + seed, [S.kpG(k) for k in range(S.Nk)], S.npw_max,
                                         S.nbands, perturb=0.15)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, :2] = np.asarray(fill)[None]
    return p, S, c_phi, c_chi, occ


def _stencil(fun, h):
    """Exact derivative at 0 of a polynomial of degree <= 4."""
    return (8 * (fun(h) - fun(-h)) - (fun(2 * h) - fun(-2 * h))) / (12 * h)


def _richardson(fun, x, h, levels=3):
    """Central differences at h, h/2, h/4 extrapolated to h -> 0 (error O(h^6))."""
    D = [(fun(x + h / 2 ** i) - fun(x - h / 2 ** i)) / (2 * h / 2 ** i) for i in range(levels)]
    for lev in range(1, levels):
        D = [(4 ** lev * D[i + 1] - D[i]) / (4 ** lev - 1) for i in range(len(D) - 1)]
    return D[0]


@pytest.mark.parametrize("A,C", PARAMS)
@pytest.mark.parametrize("wrt", ["A", "C"])
def test_kernel_derivatives_match_differences(A, C, wrt):
    """Every datum of JastrowKernels(deriv) = d/dtheta of JastrowKernels, on all three branches of B(g)."""
    g = np.array([0.05, 0.4, 0.95, 1.05, 2.5, 5.5, 6.5, 12.0, 40.0])
    p = g / C
    p2 = p * p
    Gamma0, x, Nk = 0.37, 1.0, 8

    def datum(ks, s):
        return np.concatenate([ks.u(p2, s), ks.lap(p2, s), ks.gsq(p, s), ks.gsq(np.zeros(1), s),
                               ks.V2a(p2, s), ks.V2a(p2, s, adjoint=True),
                               [ks.v0(s), ks.amp(s), ks.corr(s, Gamma0, x, Nk)]])

    for s in range(2):
        def fun(t):
            Av, Cv = np.array([0.9, 1.1]) * A, np.array([1.2, 0.8]) * C
            (Av if wrt == "A" else Cv)[s] += t
            return datum(KN.JastrowKernels(Av, Cv), s)
        Av, Cv = np.array([0.9, 1.1]) * A, np.array([1.2, 0.8]) * C
        ref = _richardson(fun, 0.0, 1e-2 * (Av if wrt == "A" else Cv)[s])
        val = datum(KN.JastrowKernels(Av, Cv, deriv=(wrt, s)), s)
        scale = np.maximum(np.abs(ref), 1e-12 * np.abs(datum(KN.JastrowKernels(Av, Cv), s)).max())
        assert np.all(np.abs(val - ref) <= 1e-9 * scale), (s, np.abs(val - ref) / scale)
        # the other channel does not depend on this parameter
        assert np.all(datum(KN.JastrowKernels(Av, Cv, deriv=(wrt, 1 - s)), s) == 0.0)


def test_energy_is_quadratic_along_the_kernel_derivative():
    """E(K + t dK) is a polynomial of degree 2 in t (corrections and ushort_factor 2 included)."""
    p, S, c_phi, c_chi, occ = tiny(seed=1, ushort_factor=2.0)
    base = KN.JastrowKernels(S.A, S.C)
    for deriv in (("C", 0), ("A", 1)):
        d = KN.JastrowKernels(S.A, S.C, deriv=deriv)
        ts = [-0.7, 0.0, 0.6, 1.3]
        Es = [OP.energy_terms(S, c_phi, c_chi, occ, kset=KN.DisplacedKernels(base, d, t))["total"] for t in ts]
        coef = np.polyfit(ts[:3], Es[:3], 2)
        assert abs(np.polyval(coef, ts[3]) - Es[3]) < 1e-11 * abs(Es[3]), deriv


@pytest.mark.parametrize("div", [1, 0])
def test_dE_dA_is_the_exact_difference_of_E(div):
    """E is quadratic in each A_s at fixed C, so the 3-point central difference is exact."""
    p, S, c_phi, c_chi, occ = tiny(seed=2, div=div)
    g = GR.param_gradient(S, c_phi, c_chi, occ)
    for s in range(2):
        h = 0.3

        def E(a):
            A = S.A.copy()
            A[s] = a
            return OP.energy_terms(make_setup(p, A=A, C=S.C, div_correction=div), c_phi, c_chi, occ)["total"]
        ref = (E(S.A[s] + h) - E(S.A[s] - h)) / (2 * h)
        assert abs(g["A"][s] - ref) < 1e-11 * max(abs(ref), 1e-3), (s, g["A"][s], ref)


@pytest.mark.parametrize("ushort_factor", [1.0, 2.0])
def test_dE_dC_matches_extrapolated_differences_of_E(ushort_factor):
    p, S, c_phi, c_chi, occ = tiny(seed=3, ushort_factor=ushort_factor)
    g = GR.param_gradient(S, c_phi, c_chi, occ)
    for s in range(2):
        def E(c):
            C = S.C.copy()
            C[s] = c
            return OP.energy_terms(make_setup(p, A=S.A, C=C, ushort_factor=ushort_factor), c_phi, c_chi,
                                   occ)["total"]
        ref = _richardson(E, S.C[s], 0.04 * S.C[s])
        assert abs(g["C"][s] - ref) < 1e-8 * abs(ref), (s, g["C"][s], ref)


@pytest.mark.parametrize("div,ushort_factor,kdep", [(1, 1.0, False), (1, 2.0, False), (0, 1.0, False),
                                                    (1, 1.0, True)])
def test_orbital_gradient_is_exact(div, ushort_factor, kdep):
    """g_phi, g_chi against the exact 4-point stencil of E along random directions (E is cubic).
    kdep: occupations that differ between the two k-points, so that a weight taken at the wrong k-point
    (f of the output k instead of the partner's, of q1 instead of q2) breaks the identity."""
    p, S, c_phi, c_chi, occ = tiny(seed=4, div=div, ushort_factor=ushort_factor, fill=(1.0, 0.55))
    if kdep:
        occ[1, :2] = (0.8, 0.35)
    g_phi, g_chi = GR.orbital_gradient(S, c_phi, c_chi, occ)
    rng = np.random.default_rng(5)
    mask = np.zeros((S.Nk, 1, S.npw_max))
    for k in range(S.Nk):
        mask[k, :, : S.npw[k]] = 1.0
    for which, g in (("phi", g_phi), ("chi", g_chi)):
        for _ in range(2):
            d = (rng.standard_normal(c_phi.shape) + 1j * rng.standard_normal(c_phi.shape)) * mask
            if which == "phi":
                fun = lambda h: OP.energy_terms(S, c_phi + h * d, c_chi, occ)["total"]
            else:
                fun = lambda h: OP.energy_terms(S, c_phi, c_chi + h * d, occ)["total"]
            ref = _stencil(fun, 1e-2)
            val = float(np.real(np.sum(np.conj(g) * d)))
            assert abs(val - ref) < 1e-10 * abs(ref), (which, val, ref)


def test_orbital_gradient_rejects_weight_outside_the_partner_bands():
    p, S, c_phi, c_chi, occ = tiny(seed=0)
    occ[:, 2] = 0.5
    with pytest.raises(ValueError):
        GR.orbital_gradient(S, c_phi, c_chi, occ)


def test_pins_detect_a_planted_mistake_in_a_derivative_kernel(monkeypatch):
    """A 3% error in d((grad u)^2)~/dC must break the dE/dC pin."""
    p, S, c_phi, c_chi, occ = tiny(seed=3)
    orig = KN.dgradu_sq_dC
    monkeypatch.setattr(KN, "dgradu_sq_dC", lambda pp, A, C: 1.03 * orig(pp, A, C))
    g = GR.param_gradient(S, c_phi, c_chi, occ)

    def E(c):
        C = S.C.copy()
        C[0] = c
        return OP.energy_terms(make_setup(p, A=S.A, C=C), c_phi, c_chi, occ)["total"]
    ref = _richardson(E, S.C[0], 0.04 * S.C[0])
    assert abs(g["C"][0] - ref) > 1e-6 * abs(ref)
