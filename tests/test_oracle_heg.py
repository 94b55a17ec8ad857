"""HEG closed forms, HF limit and BITC = TC for plane waves (pins P1, P2, P11).

For plane-wave orbitals psi_n = e^{iG_n.r} (Gamma only, chi = phi, f = 1) every
term of the operator is diagonal in momentum and its eigenvalue is a finite
lattice sum over the occupied set O, derived by hand from the algorithms
(Sec. 2.6) -- no FFT and no grid.  With D = G_n - G_m, U(D) = i D u~pp(D)/Omega,
a(q) = sum_{m in O, m != q} U(G_q - G_m), c_s = (4 pi A_s)^2 Gamma0
+ x 4 pi A_s u_short,s (N_k = 1):

  2ax  -(1/Omega) [sum_{m != n} V_2a(D) + V_J(0)] - 4 pi Gamma0/Omega
  2bx1 (1/Omega) sum_{m != n} G_m . D u~(D)
  2bx2 -(1/Omega) sum_{m != n} D . G_n u~(D)
  3a2  (1/(2 Omega^2)) sum_s [sum_{a != b} |G_a - G_b|^2 u~_s^2 + N_occ c_s]
  3a4  -sum_{q != n} a(q) . U(G_n - G_q)           (= 3b5)
  3b4  a(n) . a(n)
  3b6  (N_occ/Omega^2) sum_s [sum_{m != n} |D|^2 u~_s(D)^2 + c_s]
  all Hartree-type terms (2ah, 2bh1, 2bh2, 3a1, 3a3, 3b1, 3b2, 3b3) vanish: the
  density is uniform and G = 0 is dropped.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import kernels as KN
from oracle import operator as OP
from paper_2302_07420_gb300 import synth


def heg_case(nelec, rs, fft, radius2, radius2_occ, **kw):
    p = synth.heg_params(nelec, rs, fft, radius2)
    p.update(kw)
    S = make_setup(p, **{k: v for k, v in kw.items() if k in ("A", "C", "div_correction", "ushort_factor")})
    c = synth.heg_orbitals(S.miller[0], S.npw_max, radius2_occ)
    assert c.shape[1] == S.nocc
    occ = synth.occupations(1, S.nbands, S.nocc)
    return S, c, occ


def closed_forms(S, c):
    Om, A, C = S.Omega, S.A, S.C
    idx = [int(np.argmax(np.abs(c[0, b]))) for b in range(c.shape[1])]
    G = S.miller[0][idx] @ S.B
    no = len(G)
    div = S.div_correction

    def u(s, D):
        d2 = D @ D
        return KN.u_tilde(d2, A[s], C[s])

    def U(D):
        return 1j * D * u(0, D) / Om

    a = [sum((U(G[q] - G[m]) for m in range(no) if m != q), np.zeros(3, complex)) for q in range(no)]
    cs = [(4 * np.pi * A[s]) ** 2 * S.Gamma0 + S.ushort_factor * 4 * np.pi * A[s] * KN.u_short(A[s], C[s])
          for s in range(2)]
    e = {t: np.zeros(no, complex) for t in OP.TERMS}
    s3a2 = 0.0
    for s in range(2):
        for i in range(no):
            for j in range(no):
                if i != j:
                    D = G[i] - G[j]
                    s3a2 += (D @ D) * u(s, D) ** 2
        if div:
            s3a2 += no * cs[s]
    for n in range(no):
        v = 0.0
        for m in range(no):
            if m == n:
                continue
            D = G[n] - G[m]
            d2 = D @ D
            v += KN.V2a(d2, A[0], C[0])
            e["2bx1"][n] += (G[m] @ D) * u(0, D) / Om
            e["2bx2"][n] -= (D @ G[n]) * u(0, D) / Om
            e["3a4"][n] -= a[m] @ U(G[n] - G[m])
            e["3b6"][n] += no / Om ** 2 * sum(d2 * u(s, D) ** 2 for s in range(2))
        e["2ax"][n] = -(v + KN.V2a_jastrow_zero(A[0], C[0])) / Om - (4 * np.pi * S.Gamma0 / Om if div else 0.0)
        e["3a2"][n] = s3a2 / (2 * Om ** 2)
        e["3b4"][n] = a[n] @ a[n]
        e["3b5"][n] = e["3a4"][n]
        if div:
            e["3b6"][n] += no / Om ** 2 * sum(cs)
    return idx, e


def eigenvalues(res, c, idx):
    out = {}
    for t, v in res.items():
        ev = np.array([v[0, b, idx[b]] for b in range(len(idx))])
        off = np.abs(v[0]).sum() - np.abs(ev).sum()
        out[t] = (ev, off)
    return out


CASES = [
    dict(nelec=14, rs=4.0, fft=16, radius2=16, radius2_occ=1),                     # heg_14
    dict(nelec=38, rs=2.5, fft=15, radius2=9, radius2_occ=2),                      # 19 plane waves, odd box
    dict(nelec=14, rs=4.0, fft=16, radius2=16, radius2_occ=1, div_correction=0),
    dict(nelec=14, rs=3.0, fft=16, radius2=16, radius2_occ=1, ushort_factor=2.0),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("left", [False, True])
def test_heg_closed_forms_every_term(case, left):
    S, c, occ = heg_case(**case)
    res = OP.apply_operator(S, c, c, occ, left=left)
    idx, ref = closed_forms(S, c)
    ev = eigenvalues(res, c, idx)
    scale = max(np.abs(ref["2ax"]).max(), 1e-3)
    for t in OP.TERMS:
        val, off = ev[t]
        assert off < 1e-12 * scale, (t, off)
        if left and t in ("2ax", "2bx1", "2bx2"):
            continue     # left-operator split differs per term; the total is checked below
        np.testing.assert_allclose(val, ref[t], rtol=0, atol=1e-12 * scale, err_msg=t)
    # BITC = TC for plane waves: the left operator equals the right one (P11)
    if left:
        res_r = OP.apply_operator(S, c, c, occ, left=False)
        np.testing.assert_allclose(OP.total(res), OP.total(res_r), rtol=0, atol=1e-12 * scale)
        # and the left two-body exchange split follows V_2a^dagger and the flipped grad-u terms
        v2x = sum(ev[t][0] for t in ("2ax", "2bx1", "2bx2"))
        np.testing.assert_allclose(v2x, ref["2ax"] + ref["2bx1"] + ref["2bx2"], rtol=0, atol=1e-12 * scale)


def test_hartree_fock_limit():
    """A = 0: only 2ah + 2ax survive; HEG exchange -(4 pi/Omega) sum_{m!=n} 1/|D|^2 - c_C (P2)."""
    p = synth.heg_params(14, 4.0, 16, 16)
    S = make_setup(p, A=[0.0, 0.0])
    c = synth.heg_orbitals(S.miller[0], S.npw_max, 1)
    occ = synth.occupations(1, 7, 7)
    res = OP.apply_operator(S, c, c, occ)
    idx = [int(np.argmax(np.abs(c[0, b]))) for b in range(7)]
    G = S.miller[0][idx] @ S.B
    cC = 4 * np.pi * S.Gamma0 / S.Omega
    for t in OP.TERMS:
        if t not in ("2ax", "2ah"):
            assert np.abs(res[t]).max() == 0.0, t          # every Jastrow kernel is exactly zero
    assert np.abs(res["2ah"]).max() < 1e-30               # uniform density: Hartree vanishes
    for n in range(7):
        ex = -4 * np.pi / S.Omega * sum(1.0 / ((G[n] - G[m]) @ (G[n] - G[m])) for m in range(7) if m != n) - cC
        assert abs(res["2ax"][0, n, idx[n]] - ex) < 1e-14 * abs(ex)
