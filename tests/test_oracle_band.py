"""Pins of the band-point oracle (``oracle/band.py``): the operator at k-points off the SCF mesh.

* 4 pi Gamma_b(k)/Omega = -S(k), S(k) = sum_{R != 0} cos(k.R)/R over the Born-von Karman supercell,
  by an independent Ewald split (real and reciprocal halves both significant);
* Gamma_b and the vector sum W do not depend on alpha, W vanishes on the mesh and is odd in k;
* a band point given by a mesh point's coordinates reproduces the SCF operator there (Sec. 2.6.3: the
  SCF corrections apply on the mesh);
* HEG plane waves at an off-mesh k: every term is diagonal and equals a finite lattice sum over the
  occupied plane waves of the mesh, derived by hand from the algorithms (Sec. 2.6), plus the band
  corrections (Eqs. divcorr_2ax_band, 3b6_div_band1, divcorr_2bx1/2, div_corr_3a4_2/3, 3b5_div_2/3,
  div_corr_3b4_2/4);
* next to a mesh point (k_b = k_m + delta, delta -> 0) every term has a finite limit with the band
  corrections and diverges without them;
* the FFT route equals direct reciprocal-space sums at a band point; adjointness at the band point, which
  also fails when one member of a pair of grad-u band corrections (2bx1/2bx2, 3a3/3b3, 3a4/3b5,
  3b6 band2/band3) or a 3b4 correction has the wrong sign.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import band as BD
from oracle import cell as CL
from oracle import ewald as EW
from oracle import kernels as KN
from oracle import operator as OP
from oracle.backends import DirectBackend
from paper_2302_07420_gb300 import synth

K_OFF = np.array([0.13, 0.27, -0.31])      # fractional, off every mesh used here


@pytest.mark.parametrize("kmesh", [(1, 1, 1), (2, 2, 2), (3, 2, 1)])
@pytest.mark.parametrize("cell", ["si", "triclinic"])
def test_band_constant_is_minus_the_phased_ewald_sum(kmesh, cell):
    lat = synth.si_params()["lattice"] if cell == "si" else synth.tiny_params(3)["lattice"]
    k = K_OFF @ CL.reciprocal(lat)
    Om = abs(np.linalg.det(lat))
    gb = BD.gamma_band(lat, kmesh, CL.default_alpha(lat, kmesh), k)
    Ssc = lat * np.asarray(kmesh)[:, None]
    for eta_scale in (1.0, 0.5):
        eta = (2.2 * eta_scale / min(np.linalg.norm(Ssc, axis=1))) ** 2
        S = EW.phased_sum(Ssc, k, eta=eta)
        assert abs(4 * np.pi * gb / Om + S) < 1e-12 * max(abs(S), 1.0)


def test_band_constants_do_not_depend_on_alpha():
    lat = synth.si_params()["lattice"]
    km = (2, 2, 2)
    B = CL.reciprocal(lat)
    k = K_OFF @ B
    L = CL.shortest_supercell_vector(lat, km)
    g = [BD.gamma_band(lat, km, (L / f) ** 2, k) for f in (12, 14, 17, 20)]
    W = [BD.aux_vector_sum(lat, km, (L / f) ** 2, k) for f in (12, 14, 17, 20)]
    assert max(abs(x - g[0]) for x in g) < 1e-12 * abs(g[0])
    assert max(np.abs(w - W[0]).max() for w in W) < 1e-11 * np.abs(W[0]).max()
    assert np.abs(W[0]).max() > 1e-3                               # not trivially zero off the mesh
    a = CL.default_alpha(lat, km)
    np.testing.assert_allclose(BD.aux_vector_sum(lat, km, a, -k), -W[0], rtol=0, atol=1e-12)
    for kf in CL.kmesh_frac(km):                                   # on the mesh: odd terms cancel
        assert np.abs(BD.aux_vector_sum(lat, km, a, kf @ B)).max() < 1e-12
    with pytest.raises(ValueError):
        BD.aux_scalar_sum(lat, km, a, CL.kmesh_frac(km)[5] @ B)


def _tiny(seed, fft=(8, 9, 10), ecut=1.2, kmesh=(1, 1, 2), div=1):
    p = synth.tiny_params(seed, kmesh=kmesh, fft=fft, ecut=ecut, nbands=3, nocc=2, scale=5.0)
    S = make_setup(p, div_correction=div)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 60 + seed, [S.kpG(k) for k in range(S.Nk)],
                                         S.npw_max, S.nbands, perturb=0.2)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, 1] = 0.6
    return S, c_phi, c_chi, occ


def _band_orbitals(S, kfrac, seed, fill=0.6):
    SB = BD.BandSetup(S, kfrac)
    kp = [SB.kpG(S.Nk + i) for i in range(SB.nkb)]
    b_phi, b_chi = synth.random_orbitals(synth.SEED0 + 80 + seed, kp, SB.npw_max, S.nbands, perturb=0.2)
    b_occ = synth.occupations(SB.nkb, S.nbands, S.nocc)
    b_occ[:, 1] = fill
    return SB, b_phi, b_chi, b_occ


@pytest.mark.parametrize("left", [False, True])
def test_band_point_on_the_mesh_is_the_scf_operator(left):
    S, c_phi, c_chi, occ = _tiny(0)
    k0 = 1
    ref = OP.apply_operator(S, c_phi, c_chi, occ, left=left, kpoints=[k0])
    got = BD.band_apply(S, c_phi, c_chi, occ, S.kfrac[k0], c_phi[k0:k0 + 1], c_chi[k0:k0 + 1],
                        occ[k0:k0 + 1], left=left)
    scale = np.abs(OP.total(ref)[k0]).max()
    for t in OP.TERMS:
        np.testing.assert_allclose(got[t][0], ref[t][k0], rtol=0, atol=1e-14 * scale, err_msg=t)
    with pytest.raises(ValueError):                                # same point, shifted by a G vector
        BD.BandSetup(S, S.kfrac[k0] + np.array([1.0, 0.0, 0.0]))


@pytest.mark.parametrize("left", [False, True])
def test_fft_route_equals_direct_sums_at_a_band_point(left):
    S, c_phi, c_chi, occ = _tiny(1, fft=(6, 5, 6), ecut=1.5, kmesh=(2, 1, 1))
    SB, b_phi, b_chi, b_occ = _band_orbitals(S, K_OFF, 1)
    assert SB.on_mesh == [-1]
    a = BD.band_apply(S, c_phi, c_chi, occ, K_OFF, b_phi, b_chi, b_occ, left=left)
    b = BD.band_apply(S, c_phi, c_chi, occ, K_OFF, b_phi, b_chi, b_occ, left=left, backend=DirectBackend)
    scale = np.abs(OP.total(a)).max()
    for t in OP.TERMS:
        assert np.abs(a[t]).max() > 1e-10 * scale, t
        np.testing.assert_allclose(a[t], b[t], rtol=0, atol=1e-12 * scale, err_msg=t)


@pytest.mark.parametrize("div", [0, 1])
def test_adjointness_at_a_band_point(div):
    """<chi_i|h phi_j> = <h^dagger chi_i|phi_j> for i, j at an off-mesh band point (with its corrections)."""
    S, c_phi, c_chi, occ = _tiny(2, div=div)
    SB, b_phi, b_chi, b_occ = _band_orbitals(S, K_OFF, 2)
    r = OP.total(BD.band_apply(S, c_phi, c_chi, occ, K_OFF, b_phi, b_chi, b_occ))
    l = OP.total(BD.band_apply(S, c_phi, c_chi, occ, K_OFF, b_phi, b_chi, b_occ, left=True))
    lhs = np.conj(b_chi[0]) @ r[0].T
    rhs = np.conj(l[0]) @ b_phi[0].T
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13 * np.abs(lhs).max())


# ---------------------------------------------------------------------------------------------------
# HEG plane waves: the mesh partners are the nocc lowest |q+G|^2 at every mesh point (f = 1); the band
# point k_b carries nbands plane waves k_b + G_n, the lowest nocc of them occupied.  With
# P = q + G_m (occupied partners), D = k_b + G_n - P (never 0 off the mesh), U(D) = i D u~pp(D)/Omega,
# a(P) = (1/N_k) sum_{P'} U(P - P'), a_b(n) = (1/N_k) sum_P U(D), nbar = nocc, o_n = f_n at k_b:
#   2ax  -(1/(N_k Omega)) sum_P V_2a(D) - (4 pi Gamma_b/Omega) o_n
#   2bx1 (1/(N_k Omega)) sum_P P.D u~(D)          2bx2  -(1/(N_k Omega)) sum_P D.(k_b + G_n) u~(D)
#   3a4 = 3b5  -(1/N_k) sum_P a(P).U(D)           3b4   a_b(n).a_b(n)
#   3b6  (nbar/(N_k Omega^2)) sum_P sum_s |D|^2 u~_s(D)^2 + (nbar/Omega^2) sum_s (4 pi A_s)^2 Gamma_b o_n
#   3a2  the SCF operator's value (h6 is a partner-only, uniform field)
#   Hartree-type terms vanish (uniform density, G = 0 dropped).
# Grad-u band corrections (c = 4 pi A_pp/(N_k Omega), W = W(k_b), K_n = k_b + G_n): 2bx1 gains
# -c (W.K_n) o_n and 2bx2 +c (W.K_n) o_n; 3a4 and 3b5 gain i c o_n (W.a_b(n)) + c^2 o_n^2 (W.W) (the band
# point's own h3 fields are (a_b(n) - i c W o_n) e^{iG_n.r} and (-a_b(n) + i c W o_n) e^{-iG_n.r});
# 3b4 becomes a_b.a_b - 2 i c o_n (W.a_b) - c^2 o_n^2 (W.W); those of 3a3, 3b3 and 3b6 (band2/3) vanish
# (h1 = 0, and n~ has only its G = 0 component).
# ---------------------------------------------------------------------------------------------------

def _near_mesh(div, deltas, general=False, m=1):
    """Band operator at k_b = k_m + delta e next to the mesh point k_m, with k_m's own orbitals as the band
    point's (its sphere is the same for these delta), A_pp != A_ap.  general: left orbitals that are not
    biorthonormal to the right ones (the general-overlap forms) and occupations that differ between
    k-points."""
    p = synth.tiny_params(2, kmesh=(1, 1, 2), fft=(8, 9, 10), ecut=1.2, nbands=3, nocc=2, scale=5.0)
    S = make_setup(p, A=[p["A"][0], 1.6 * p["A"][0]], div_correction=div)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 62, [S.kpG(k) for k in range(S.Nk)], S.npw_max,
                                         S.nbands, perturb=0.2)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, 1] = 0.6
    if general:
        rng = np.random.default_rng(synth.SEED0 + 63)
        for k in range(S.Nk):
            n = S.npw[k]
            c_chi[k, :, :n] += 0.15 * (rng.standard_normal((S.nbands, n)) + 1j * rng.standard_normal((S.nbands, n)))
        occ[m, 1] = 0.85
    e = np.array([0.31, -0.52, 0.79])
    e /= np.linalg.norm(e)
    out = []
    for d in deltas:
        # the point next to k_m, and a second band point far from the mesh whose outputs must not
        # depend on the first (its own Gamma_b, W and orbitals)
        kb = np.stack([S.kfrac[m] + d * e, K_OFF])
        SB = BD.BandSetup(S, kb)
        assert np.array_equal(SB.miller[S.Nk], S.miller[m])
        bp, bc = synth.random_orbitals(synth.SEED0 + 64, [SB.kpG(S.Nk + 1)], SB.npw_max, S.nbands, perturb=0.2)
        n0 = S.npw[m]
        b_phi = np.zeros((2, S.nbands, SB.npw_max), complex)
        b_chi = np.zeros_like(b_phi)
        b_phi[0, :, :n0], b_chi[0, :, :n0] = c_phi[m, :, :n0], c_chi[m, :, :n0]
        b_phi[1], b_chi[1] = bp[0], bc[0]
        b_occ = np.stack([occ[m], occ[m]])
        out.append(BD.band_apply(S, c_phi, c_chi, occ, kb, b_phi, b_chi, b_occ))
    return out


@pytest.mark.parametrize("general", [False, True])
def test_band_corrections_cancel_the_singularity_next_to_a_mesh_point(general):
    """Off the mesh every q + G is kept in the sums, and the partner q = k_m enters with the kernel at
    p = k_b - k_m, which diverges as k_b -> k_m: 4 pi/p^2 in 2ax and, through U U, in 3b6; i p u~(p) ~ 1/p
    in the grad-u terms.  The band corrections (Gamma_b of Eq. divcorr_2ax_band and 3b6_div_band1, the
    vector sum W of Eq. correction_nabla in the grad-u and 3b6 band2/3 forms) carry the same singular
    parts with the opposite sign, so with them every term has a finite limit; without them the terms
    grow as 1/delta or 1/delta^2.  A wrong sign or amplitude of any correction (W, Gamma_b, A_pp against
    A_ap) leaves a divergent remainder."""
    near = _near_mesh(1, (1e-3, 1e-4), general)
    bare = _near_mesh(0, (1e-3, 1e-4), general)
    scale = max(np.abs(near[0][t][0]).max() for t in OP.TERMS)
    for t in OP.TERMS:
        a, b = near[0][t][0], near[1][t][0]
        assert np.abs(b - a).max() <= 0.02 * max(np.abs(a).max(), 1e-3 * scale), t
        far = np.abs(near[0][t][1]).max()
        assert np.abs(near[1][t][1] - near[0][t][1]).max() <= 1e-12 * max(far, scale), t   # the far point
    for t in ("2ax", "2bx1", "2bx2", "3a3", "3a4", "3b3", "3b4", "3b5", "3b6"):
        assert np.abs(bare[1][t][0]).max() > 5.0 * np.abs(bare[0][t][0]).max(), t  # the singular terms are there


def _heg_band_case(kmesh=(2, 2, 1), nbands=9, A=None):
    p = synth.heg_params(14, 4.0, 12, 4)
    p["kmesh"] = kmesh
    p["nbands"] = nbands
    kw = {} if A is None else dict(A=A)
    S = make_setup(p, **kw)
    c = synth.heg_kpoint_orbitals([S.kpG(k) for k in range(S.Nk)], S.miller, S.npw_max, nbands)
    occ = synth.occupations(S.Nk, nbands, S.nocc)
    SB = BD.BandSetup(S, K_OFF)
    cb = synth.heg_kpoint_orbitals([SB.kpG(S.Nk)], [SB.miller[S.Nk]], SB.npw_max, nbands)
    occ_b = synth.occupations(1, nbands, S.nocc)
    return S, SB, c, occ, cb, occ_b


def _heg_band_closed_forms(S, SB, c, cb, occ_b):
    Om, A, C, Nk, no = S.Omega, S.A, S.C, S.Nk, S.nocc
    P = np.array([S.kpG(k)[int(np.argmax(np.abs(c[k, b])))] for k in range(Nk) for b in range(no)])
    idx = [int(np.argmax(np.abs(cb[0, b]))) for b in range(cb.shape[1])]
    Kn = SB.kpG(Nk)[idx]
    gb = SB.gamma_b[0]

    def u(s, D):
        return KN.u_tilde(np.einsum("...i,...i->...", D, D), A[s], C[s])

    def U(D):
        return 1j * D * u(0, D)[..., None] / Om

    a = np.array([U(P[i] - np.delete(P, i, axis=0)).sum(axis=0) / Nk for i in range(len(P))])
    e = {t: np.zeros(len(idx), complex) for t in OP.TERMS}
    for n in range(len(idx)):
        D = Kn[n] - P
        d2 = np.einsum("ij,ij->i", D, D)
        o = occ_b[0, n] if n < no else 0.0
        e["2ax"][n] = -KN.V2a(d2, A[0], C[0]).sum() / (Nk * Om) - 4 * np.pi * gb / Om * o
        cW = 4 * np.pi * A[0] / (Nk * Om) * (SB.W[0] @ Kn[n]) * o
        e["2bx1"][n] = np.einsum("ij,ij->i", P, D) @ u(0, D) / (Nk * Om) - cW
        e["2bx2"][n] = -(D @ Kn[n]) @ u(0, D) / (Nk * Om) + cW
        ab = U(D).sum(axis=0) / Nk
        c = 4 * np.pi * A[0] / (Nk * Om)
        W = SB.W[0]
        e["3b4"][n] = ab @ ab - 2j * c * o * (W @ ab) - (c * o) ** 2 * (W @ W)
        e["3a4"][n] = -np.einsum("ij,ij->", a, U(D)) / Nk + 1j * c * o * (W @ ab) + (c * o) ** 2 * (W @ W)
        e["3b5"][n] = e["3a4"][n]
        e["3b6"][n] = (no / (Nk * Om ** 2)) * sum(d2 @ u(s, D) ** 2 for s in range(2)) \
            + (no / Om ** 2) * sum((4 * np.pi * A[s]) ** 2 for s in range(2)) * gb * o
    return idx, e


@pytest.mark.parametrize("A", [None, [0.0, 0.0]])
def test_heg_closed_forms_off_the_mesh(A):
    S, SB, c, occ, cb, occ_b = _heg_band_case(A=A)
    res = BD.band_apply(S, c, c, occ, K_OFF, cb, cb, occ_b)
    idx, ref = _heg_band_closed_forms(S, SB, c, cb, occ_b)
    scf3a2 = OP.apply_operator(S, c, c, occ, kpoints=[0], terms=("3a2",))["3a2"]
    i0 = int(np.argmax(np.abs(c[0, 0])))
    ref["3a2"][:] = scf3a2[0, 0, i0]
    scale = np.abs(ref["2ax"]).max()
    for t in OP.TERMS:
        v = res[t][0]
        ev = np.array([v[b, idx[b]] for b in range(len(idx))])
        assert np.abs(v).sum() - np.abs(ev).sum() < 1e-12 * scale, t        # diagonal
        np.testing.assert_allclose(ev, ref[t], rtol=0, atol=1e-12 * scale, err_msg=t)
    # BITC = TC for plane waves at the band point too
    left = OP.total(BD.band_apply(S, c, c, occ, K_OFF, cb, cb, occ_b, left=True))
    np.testing.assert_allclose(left, OP.total(res), rtol=0, atol=1e-12 * scale)


def test_band_pins_detect_a_planted_mistake(monkeypatch):
    """A band point that took the SCF constant Gamma0 instead of Gamma_b fails the closed forms."""
    S, SB, c, occ, cb, occ_b = _heg_band_case(A=[0.0, 0.0])
    _, ref = _heg_band_closed_forms(S, SB, c, cb, occ_b)
    monkeypatch.setattr(BD, "gamma_band", lambda lat, km, al, k: CL.gamma0(lat, km, al))
    res = BD.band_apply(S, c, c, occ, K_OFF, cb, cb, occ_b)
    idx = [int(np.argmax(np.abs(cb[0, b]))) for b in range(cb.shape[1])]
    ev = np.array([res["2ax"][0, b, idx[b]] for b in range(len(idx))])
    assert np.abs(ev - ref["2ax"]).max() > 1e-4 * np.abs(ref["2ax"]).max()


@pytest.mark.parametrize("pair", ["2bx", "3a3b3", "3a4b5", "3b4", "3b6"])
def test_adjointness_catches_a_sign_error_in_each_corrected_pair(pair, monkeypatch):
    """Each pair of grad-u band corrections is adjoint to itself as a pair: flipping one member breaks
    <chi_i|h phi_j> = <h^dagger chi_i|phi_j> at the band point."""
    S, c_phi, c_chi, occ = _tiny(2)
    SB, b_phi, b_chi, b_occ = _band_orbitals(S, K_OFF, 2)
    if pair == "3b6":
        orig = BD.BandOperator._corr_3b6

        def band3(self, k):
            # the band3 part of the 3b6 correction alone (Eq. 3b6_div_band3, oracle normalisation)
            S_, bk = self.S, self.bk
            no, Om = S_.nocc, S_.Omega
            WG = np.einsum("...i,i->...", S_.Gbox, S_.W[k - S_.Nk])
            F = bk.FT(bk.mul(bk.conj(self.bra[k][:no])[:, None], self.ket[k][None]))
            out = bk.zeros((S_.nbands,))
            for s_ in range(2):
                a = 4 * np.pi * self.ks.amp(s_) / S_.Nk
                X3 = np.sum(WG * self.us[s_] * F * bk.spec_neg(self.nt), axis=(-3, -2, -1))
                for q in range(no):
                    field = -a * X3[q][:, None, None, None] * bk.const(1.0)[None]
                    out = out + self.f[k][q] * bk.mul(self.ket[k][q][None], field) / (Om * Om)
            return out

        def flipped(self, k):
            return orig(self, k) - 2.0 * band3(self, k)      # band3 with the wrong sign
        monkeypatch.setattr(BD.BandOperator, "_corr_3b6", flipped)
    else:
        orig = BD.BandOperator._corr_gradu_band

        def flipped(self, k, acc):
            if pair == "3b4":
                # the 3b4 correction is adjoint to itself as a whole; its w_j part (Eq. div_corr_3b4_2) and
                # Eq. div_corr_3b4_4 are each other's adjoint: flip the sign of the w_j part only
                acc = orig(self, k, acc)
                S_, no = self.S, self.S.nocc
                c = 4 * np.pi * self.ks.amp(0) / (S_.Nk * S_.Omega)
                wc = -1j * c * np.einsum("d,mj,m...->jd...", S_.W[k - S_.Nk], self.f[k][:, None] * self._overlaps(k),
                                         self.ket[k][:no])
                acc["3b4"] = acc["3b4"] + 2.0 * self._pass_3b4(k, wc)
                return acc
            term = {"2bx": "2bx2", "3a3b3": "3b3", "3a4b5": "3b5"}[pair]
            before = acc[term].copy()
            acc = orig(self, k, acc)
            acc[term] = 2 * before - acc[term]      # this member's correction with the wrong sign
            return acc
        monkeypatch.setattr(BD.BandOperator, "_corr_gradu_band", flipped)
    r = OP.total(BD.band_apply(S, c_phi, c_chi, occ, K_OFF, b_phi, b_chi, b_occ))
    l = OP.total(BD.band_apply(S, c_phi, c_chi, occ, K_OFF, b_phi, b_chi, b_occ, left=True))
    lhs = np.conj(b_chi[0]) @ r[0].T
    rhs = np.conj(l[0]) @ b_phi[0].T
    assert np.abs(lhs - rhs).max() > 1e-9 * np.abs(lhs).max()
