"""Value pins of the Hartree-type terms for a non-uniform density (Gamma only).

The HEG closed forms make every Hartree-type term vanish (uniform density,
G = 0 dropped), so they cannot see how the oracle sums the spin channels of
the Hartree-type kernels.  Here the orbitals are a few plane waves with
random complex coefficients (Gamma only, one k-point), so the density has a
finite number of Fourier components G != 0 and every term is a finite lattice
sum over those components.  The sums are evaluated below in reciprocal space
on sparse coefficient maps {Miller vector: coefficient}: a product of two
fields is the convolution of their maps, a kernel multiplies each component
by its value at G, and no grid or FFT is involved.  The box is chosen so that
no product of the oracle's grid route wraps around (every intermediate stays
within Miller index 5 of a 16^3 box), where the discrete operator equals these
sums.

Spin structure (Sec. 2.6.3 after Alg. 1; Algs. 3, 7, 8; Eqs. 3b6_div_scf2/3
and divcor_3a2_second): an electron of spin sigma feels the Hartree-type
fields of both spin densities, n_up = n_down = n for a non-polarised state,
through the parallel-spin kernel (A, C_pp) for sigma' = sigma and the
antiparallel one (A, C_ap) for sigma' != sigma.  So every Hartree-type kernel
is the channel sum
    V_h(G) = [V_2a(G; A, C_pp) + V_2a(G; A, C_ap)] / Omega,
    u_h(G) = [u~(G; A, C_pp) + u~(G; A, C_ap)] / Omega,   U_h(G) = i G u_h(G),
while exchange-type kernels pair same-spin orbitals only, U_pp(G) = i G u~(G; A, C_pp)/Omega.
With C_pp = sqrt(2A) != C_ap = sqrt(A) (cusp conditions) a mistake in that sum
changes every Hartree-type value; the last test plants such mistakes in the
oracle and checks that they fail.

Terms (right operator; s = +1; the left operator swaps phi and chi, uses
V_2a^dagger and s = -1), with n = sum_q f chi_q^* phi_q, m = sum_q f chi_q^*
grad phi_q, h1 = FT^-1[U_h n~] (G != 0):
  2ah   FT^-1[V_h n~] phi_j                       (Alg. 1)
  2bh1  s h1 . grad phi_j                          (Sec. 2.6.3)
  2bh2  s FT^-1[-U_h . m~] phi_j                   (Sec. 2.6.3)
  3a1   -(1/2) (h1 . h1) phi_j                     (Alg. 3)
  3a3   h1 . w_j,  w_j = sum_q f phi_q FT^-1[U_pp FT[chi_q^* phi_j]]       (Alg. 5, x2)
  3b1   -FT^-1[-U_h . FT[h1 n]] phi_j              (Alg. 7, x2)
  3b2   FT^-1[-U_h . FT[h5]] phi_j, h5 = sum_q2 f h3b(q2) phi_q2,
        h3b(q2) = sum_q1 f FT^-1[U_pp FT[chi_q2^* phi_q1]] chi_q1^*       (Alg. 8, x2)
  3b3   sum_q f phi_q FT^-1[-U_pp . FT[h1 chi_q^* phi_j]]                 (Alg. 9, x2)
and the divergence corrections that carry a per-channel u~_s (G != 0):
  3a2   (1/2) phi_j sum_q2 f_q2/Omega^2 sum_s (4 pi A_s) FT^-1[u~_s (F_a + F_b)]
        (Eq. divcor_3a2_second, general-overlap form; the constant part c_s F0
        is pinned by the HEG closed forms)
  3b6   sum_q f phi_q /Omega^2 sum_s (4 pi A_s) [O_qj FT^-1[u~_s n~] + X_s,qj]
        (Eqs. 3b6_div_scf2/3, times the multiplicity 2 of 3b and the 1/2 of 3b6)
"""
from collections import defaultdict

import numpy as np
import pytest

from conftest import make_setup
from oracle import kernels as KN
from oracle import operator as OP
from paper_2302_07420_gb300 import synth

HARTREE_TERMS = ("2ah", "2bh1", "2bh2", "3a1", "3a3", "3b1", "3b2", "3b3")
SUPPORT = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


# ----------------------------------------------------------------- sparse maps
def _add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def mul(a, b):
    out = defaultdict(complex)
    for ma, va in a.items():
        for mb, vb in b.items():
            out[_add(ma, mb)] += va * vb
    return dict(out)


def conj(a):
    return {(-m[0], -m[1], -m[2]): np.conj(v) for m, v in a.items()}


def lin(*pairs):
    out = defaultdict(complex)
    for s, a in pairs:
        for m, v in a.items():
            out[m] += s * v
    return dict(out)


class Cell:
    def __init__(self, S):
        self.S = S
        self.B = S.B
        self.Om = S.Omega

    def G(self, m):
        return np.asarray(m, dtype=np.float64) @ self.B

    def g2(self, m):
        g = self.G(m)
        return float(g @ g)

    def grad(self, a, d):
        return {m: 1j * self.G(m)[d] * v for m, v in a.items()}

    def kern(self, a, fn):
        """Component-wise kernel fn(m) (fn returns 0 where the kernel is dropped)."""
        return {m: fn(m) * v for m, v in a.items()}


def _nonzero(fn):
    def f(m):
        return 0.0 if m == (0, 0, 0) else fn(m)
    return f


def closed_forms(S, phi, chi, f, left=False):
    """Per-term outputs {term: [per band: sparse map]} of the Hartree-type terms and of the
    u~_s parts of the 3a2 / 3b6 corrections, from the finite lattice sums above."""
    cl = Cell(S)
    A, C, Om = S.A, S.C, S.Omega
    sgn = -1.0 if left else 1.0
    ket, bra = (chi, phi) if left else (phi, chi)
    nb, no = len(ket), len(f)

    # kernels; Hartree-type: both spin channels, exchange-type: parallel spins only
    def Vh(m):
        return sum(KN.V2a(cl.g2(m), A[s], C[s], adjoint=left) for s in range(2)) / Om

    def uh(m):
        return sum(KN.u_tilde(cl.g2(m), A[s], C[s]) for s in range(2)) / Om

    def Uh(d):
        return _nonzero(lambda m: 1j * cl.G(m)[d] * uh(m))

    def Upp(d):
        return _nonzero(lambda m: 1j * cl.G(m)[d] * KN.u_tilde(cl.g2(m), A[0], C[0]) / Om)

    def us(s):
        return _nonzero(lambda m: KN.u_tilde(cl.g2(m), A[s], C[s]))

    n = lin(*[(f[q], mul(conj(bra[q]), ket[q])) for q in range(no)])
    mvec = [lin(*[(f[q], mul(conj(bra[q]), cl.grad(ket[q], d))) for q in range(no)]) for d in range(3)]
    vH = cl.kern(n, _nonzero(Vh))
    h1 = [cl.kern(n, Uh(d)) for d in range(3)]
    vb2 = lin(*[(-1.0, cl.kern(mvec[d], Uh(d))) for d in range(3)])
    h1h1 = lin(*[(1.0, mul(h1[d], h1[d])) for d in range(3)])
    t3b1 = lin(*[(-1.0, cl.kern(mul(h1[d], n), Uh(d))) for d in range(3)])
    h3b = [[lin(*[(f[q1], mul(cl.kern(mul(conj(bra[q2]), ket[q1]), Upp(d)), conj(bra[q1])))
                  for q1 in range(no)]) for d in range(3)] for q2 in range(no)]
    h5 = [lin(*[(f[q2], mul(h3b[q2][d], ket[q2])) for q2 in range(no)]) for d in range(3)]
    t3b2 = lin(*[(-1.0, cl.kern(h5[d], Uh(d))) for d in range(3)])

    out = {t: [] for t in HARTREE_TERMS + ("3a2_us", "3b6_us")}
    # 3a2 correction, u~_s part (general overlaps): O[a][b] = <chi_a|phi_b> for the bra/ket roles
    O = [[mul(conj(bra[a]), ket[b]).get((0, 0, 0), 0.0) for b in range(nb)] for a in range(no)]
    h6u = {}
    for q2 in range(no):
        Fa = lin(*[(f[q1] * O[q1][q2], mul(conj(bra[q2]), ket[q1])) for q1 in range(no)])
        Fb = lin(*[(f[q1] * O[q2][q1], mul(conj(bra[q1]), ket[q2])) for q1 in range(no)])
        for s in range(2):
            field = cl.kern(lin((1.0, Fa), (1.0, Fb)), us(s))
            h6u = lin((1.0, h6u), (f[q2] * 4 * np.pi * A[s] / Om ** 2, field))
    for j in range(nb):
        kj = ket[j]
        gk = [cl.grad(kj, d) for d in range(3)]
        out["2ah"].append(mul(vH, kj))
        out["2bh1"].append(lin(*[(sgn, mul(h1[d], gk[d])) for d in range(3)]))
        out["2bh2"].append(lin((sgn, mul(vb2, kj))))
        out["3a1"].append(lin((-0.5, mul(h1h1, kj))))
        w = [lin(*[(f[q], mul(ket[q], cl.kern(mul(conj(bra[q]), kj), Upp(d)))) for q in range(no)])
             for d in range(3)]
        out["3a3"].append(lin(*[(1.0, mul(h1[d], w[d])) for d in range(3)]))
        out["3b1"].append(lin((-1.0, mul(t3b1, kj))))
        out["3b2"].append(mul(t3b2, kj))
        t3b3 = [lin(*[(-1.0, cl.kern(mul(h1[d], mul(conj(bra[q]), kj)), Upp(d))) for d in range(3)])
                for q in range(no)]
        out["3b3"].append(lin(*[(f[q], mul(ket[q], t3b3[q])) for q in range(no)]))
        out["3a2_us"].append(lin((0.5, mul(h6u, kj))))
        c3b6 = {}
        for q in range(no):
            F = mul(conj(bra[q]), kj)
            Oqj = F.get((0, 0, 0), 0.0)
            for s in range(2):
                vu = cl.kern(n, us(s))
                X = sum(us(s)(m) * v * n.get((-m[0], -m[1], -m[2]), 0.0) for m, v in F.items())
                field = lin((Oqj, vu), (X, {(0, 0, 0): 1.0}))
                c3b6 = lin((1.0, c3b6), (f[q] * 4 * np.pi * A[s] / Om ** 2, mul(ket[q], field)))
        out["3b6_us"].append(c3b6)
    return out


# ----------------------------------------------------------------- inputs
def make_case(left_perturb=0.15, seed=7):
    p = synth.heg_params(14, 3.0, 16, 16)
    # A_ap != A_pp (the API takes both channels' A and C independently), so that a mix-up of
    # the channels in the per-channel correction fields changes their values too
    A = [p["A"][0], 0.8 * p["A"][1]]
    S = make_setup(p, nbands=3, nocc=2, A=A)
    rng = np.random.default_rng(synth.SEED0 + 900 + seed)
    nb = 3
    P = rng.standard_normal((len(SUPPORT), nb)) + 1j * rng.standard_normal((len(SUPPORT), nb))
    Q, _ = np.linalg.qr(P)
    R = rng.standard_normal((len(SUPPORT), nb)) + 1j * rng.standard_normal((len(SUPPORT), nb))
    X = Q + left_perturb * R / np.linalg.norm(R, axis=0, keepdims=True)
    phi = [{m: complex(Q[i, b]) for i, m in enumerate(SUPPORT)} for b in range(nb)]
    chi = [{m: complex(X[i, b]) for i, m in enumerate(SUPPORT)} for b in range(nb)]
    f = np.array([1.0, 0.7])
    return S, phi, chi, f


def to_coeffs(S, maps):
    mil = [tuple(int(x) for x in m) for m in S.miller[0]]
    pos = {m: i for i, m in enumerate(mil)}
    c = np.zeros((1, len(maps), S.npw_max), dtype=np.complex128)
    for b, mp in enumerate(maps):
        for m, v in mp.items():
            c[0, b, pos[m]] = v
    return c


def on_sphere(S, maps):
    """Sparse maps -> sphere coefficients (components outside the sphere are not outputs)."""
    mil = [tuple(int(x) for x in m) for m in S.miller[0]]
    out = np.zeros((1, len(maps), S.npw_max), dtype=np.complex128)
    for b, mp in enumerate(maps):
        for i, m in enumerate(mil):
            out[0, b, i] = mp.get(m, 0.0)
    return out


def oracle_outputs(S, phi, chi, f, left):
    occ = np.zeros((1, S.nbands))
    occ[0, : len(f)] = f
    c_phi, c_chi = to_coeffs(S, phi), to_coeffs(S, chi)
    return OP.apply_operator(S, c_phi, c_chi, occ, left=left)


def compare(S, phi, chi, f, left, div):
    """Max relative deviation per checked quantity between the oracle and the lattice sums."""
    ref = closed_forms(S, phi, chi, f, left=left)
    res = oracle_outputs(S, phi, chi, f, left)
    dev = {}
    for t in HARTREE_TERMS:
        exp = on_sphere(S, ref[t])
        scale = max(np.abs(exp).max(), 1e-300)
        dev[t] = float(np.abs(res[t] - exp).max() / scale)
    if div:
        S0 = make_setup_from(S, div_correction=0)
        res0 = oracle_outputs(S0, phi, chi, f, left)
        for t in ("3a2", "3b6"):
            exp = on_sphere(S, ref[t + "_us"])
            # the constant parts c_s F0 / c_s n0 O of the corrections are added to the u~_s parts
            const = constant_corrections(S, phi, chi, f, left, t)
            got = res[t] - res0[t] - const
            dev[t + "_us"] = float(np.abs(got - exp).max() / np.abs(exp).max())
    return dev, ref


def make_setup_from(S, **kw):
    from oracle.cell import Setup
    args = dict(lattice=S.lattice, kmesh=S.kmesh, ecut=S.ecut, fft=S.n, nbands=S.nbands, nocc=S.nocc,
                A=S.A, C=S.C, alpha=S.alpha, div_correction=S.div_correction, ushort_factor=S.ushort_factor)
    args.update(kw)
    return Setup(**args)


def constant_corrections(S, phi, chi, f, left, term):
    """The constant parts of the corrections (c_s = (4 pi A_s)^2 Gamma0 + x 4 pi A_s u_short,s):
    3a2: (1/2) phi_j sum_q2 f_q2 sum_s c_s F0(q2)/Omega^2;  3b6: sum_q f phi_q sum_s c_s n~(0) O_qj/Omega^2."""
    ket, bra = (chi, phi) if left else (phi, chi)
    nb, no = len(ket), len(f)
    A, C, Om = S.A, S.C, S.Omega
    cs = sum((4 * np.pi * A[s]) ** 2 * S.Gamma0 + S.ushort_factor * 4 * np.pi * A[s] * KN.u_short(A[s], C[s])
             for s in range(2))
    O = [[mul(conj(bra[a]), ket[b]).get((0, 0, 0), 0.0) for b in range(nb)] for a in range(no)]
    outs = []
    if term == "3a2":
        F0 = sum(f[q2] * sum(f[q1] * O[q2][q1] * O[q1][q2] for q1 in range(no)) for q2 in range(no))
        for j in range(nb):
            outs.append({m: 0.5 * cs * F0 / Om ** 2 * v for m, v in ket[j].items()})
    else:
        n0 = sum(f[q] * O[q][q] for q in range(no))
        for j in range(nb):
            outs.append(lin(*[(f[q] * cs * n0 * O[q][j] / Om ** 2, ket[q]) for q in range(no)]))
    return on_sphere(S, outs)


# ----------------------------------------------------------------- tests
@pytest.mark.parametrize("left", [False, True])
@pytest.mark.parametrize("div", [0, 1])
def test_hartree_terms_match_lattice_sums(left, div):
    S, phi, chi, f = make_case()
    if not div:
        S = make_setup_from(S, div_correction=0)
    dev, ref = compare(S, phi, chi, f, left, div)
    for t, d in dev.items():
        assert d < 1e-11, (t, d)
    # the case has power: each Hartree-type output is a sizeable, non-diagonal field
    for t in HARTREE_TERMS:
        assert max(np.abs(on_sphere(S, ref[t])).max(), 0) > 1e-6, t


def test_density_is_not_uniform():
    S, phi, chi, f = make_case()
    n = lin(*[(f[q], mul(conj(chi[q]), phi[q])) for q in range(len(f))])
    assert sum(abs(v) for m, v in n.items() if m != (0, 0, 0)) > 0.1
    assert abs(S.C[0] - S.C[1]) > 0.1 and abs(S.A[0] - S.A[1]) > 0.1   # the channels differ


def _planted_channels(mode):
    """Copies of TCOperator.hartree_kernels with a planted mistake in the spin-channel sum."""
    def hk(self):
        S = self.S
        G = S.Gbox
        g2 = np.einsum("...i,...i->...", G, G)
        zero = g2 == 0.0
        g2s = np.where(zero, 1.0, g2)
        ks = self.ks
        if mode == "ap_dropped_pp_doubled":
            Vh = 2.0 * ks.V2a(g2s, 0, adjoint=self.left)
            uh = 2.0 * ks.u(g2s, 0)
            us = [np.where(zero, 0.0, ks.u(g2s, s)) for s in range(2)]
        elif mode == "pp_only":
            Vh = ks.V2a(g2s, 0, adjoint=self.left)
            uh = ks.u(g2s, 0)
            us = [np.where(zero, 0.0, ks.u(g2s, s)) for s in range(2)]
        else:   # "us_channels_swapped": the per-channel fields of the corrections exchanged
            Vh = sum(ks.V2a(g2s, s, adjoint=self.left) for s in range(2))
            uh = sum(ks.u(g2s, s) for s in range(2))
            us = [np.where(zero, 0.0, ks.u(g2s, 1 - s)) for s in range(2)]
        Vh = np.where(zero, 0.0, Vh) / S.Omega
        uh = np.where(zero, 0.0, uh) / S.Omega
        Uh = 1j * np.moveaxis(G, -1, 0) * uh[None]
        return Vh, Uh, us
    return hk


@pytest.mark.parametrize("mode", ["ap_dropped_pp_doubled", "pp_only", "us_channels_swapped"])
def test_planted_channel_mistakes_fail(monkeypatch, mode):
    S, phi, chi, f = make_case()
    monkeypatch.setattr(OP.TCOperator, "hartree_kernels", _planted_channels(mode))
    dev, _ = compare(S, phi, chi, f, left=False, div=1)
    bad = [t for t, d in dev.items() if d > 1e-6]
    if mode == "us_channels_swapped":
        assert set(bad) >= {"3a2_us", "3b6_us"}, dev
    else:
        assert set(bad) >= set(HARTREE_TERMS), dev
