"""Band-structure (off-mesh) k-points of the TC operator (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.6.3 (after Eq. divcorr_2ax_scf) and Sec. 2.6.4 (3b6): a band k-point
k_b carries output orbitals, and its own occupied orbitals as a non-SCF
calculation at k_b provides them, but it is not a partner.  Every sum over
occupied q runs over the SCF mesh, and every partner-only field (densities,
Hartree-type fields, the occupied-pair stage h3 and h6 with its 3a2
correction) is that of the SCF operator.  The pair terms take their kernels at
k_b - q + G, which for k_b off the mesh is never zero.

Divergence corrections.  A band point that coincides with a mesh point takes
the SCF corrections, as the paper states; give such a point by the mesh
point's own fractional coordinates.  Off the mesh no term is excluded from the
sums, so the finite limits of an excluded term (the -alpha of Eq. correction2,
u_short) drop out and the auxiliary sum runs over every q and G:

  Gamma_b(k) = Omega/(4 sqrt(pi^3 alpha)) - (1/N_k) sum_{q,G} A_aux(k - q + G),

the band counterpart of Gamma0 (Eq. correction).  With it:

  2ax  Eq. divcorr_2ax_band: -(4 pi Gamma_b/Omega) sum_mu f_mu <bra_mu|ket_j> ket_mu over the
       band point's own occupied orbitals mu (the SCF correction with Gamma0 -> Gamma_b);
  3b6  Eq. 3b6_div_band1: the scf1 form with (4 pi A)^2 Gamma0 + x 4 pi A u_short/N_k replaced
       by (4 pi A)^2 Gamma_b.

The grad-u terms have odd singular parts, U(p) ~ i (4 pi A/Omega) p/p^2, and
Eq. correction_nabla adds -(1/N_k) W(k) . F(0) to a sum (1/N_k) sum (p/p^2) F,
with the vector sum

  W(k) = sum_{q,G} (k - q + G) A_aux(k - q + G)

(``aux_vector_sum``; zero on the mesh).  With c = 4 pi A_pp/(N_k Omega),
O_mj = <bra_m|ket_j> and the band point's own occupied m:

  2bx1  Eq. divcorr_2bx1:  + s i c sum_m f_m O_mj (W . grad ket_m)
  2bx2  Eq. divcorr_2bx2:  - s i c sum_m f_m (W . <bra_m|grad ket_j>) ket_m
  3a3   Eq. divcorr_3a3 (on w_j, times h1):  - i c sum_m f_m O_mj (h1 . W) ket_m
  3b3   Eq. div_corr_3b3_2:  + i c sum_m f_m (W . <bra_m|h1 ket_j>) ket_m
  3b6   Eqs. 3b6_div_band2/3 (multiplicity 2 times 1/2):
        - (4 pi A_s/N_k) [O_mj FT^{-1}[(W.G) u~_s n~] + sum_{G != 0} (W.G) u~_s(G) FT[bra_m^* ket_j](G) n~(-G)]
        times f_m ket_m / Omega^2,

  3a4   Eqs. div_corr_3a4_2/3:  + i c sum_m f_m O_mj (W . h3a(m))
  3b5   Eqs. 3b5_div_2/3:  - i c sum_m f_m (W . FT[ket_j h3b(m)](0)) ket_m
  3b4   Eq. div_corr_3b4_2 (w_j -> w_j + w_c, w_c = -i c W sum_m f_m O_mj ket_m, the
        3a3 correction) and Eq. div_corr_3b4_4: - i c sum_m f_m (W . <bra_m|w_j + w_c>) ket_m,

s = +1 right, -1 left (the sign of the grad u . grad terms), where h3a(m),
h3b(m) are the occupied-pair fields of the band point's own occupied orbitals
(``_band_h3``), themselves corrected for q1 -> k_b, which gives the W . W terms
of Eqs. div_corr_3a4_3 and 3b5_div_3.  The pairs (2bx1, 2bx2), (3a3, 3b3),
(3a4, 3b5) and (3b6 band2, band3) are each adjoint to each other and the 3b4
corrections to themselves, so <chi_i|h phi_j> = <h^dagger chi_i|phi_j> holds
with them and fails if one sign of a pair is wrong.

Pins: tests/test_oracle_band.py (4 pi Gamma_b/Omega against an independent
phased Ewald sum, alpha-independence of Gamma_b and W, a band point on the
mesh reproduces the SCF operator, HEG closed forms off the mesh, direct sums,
adjointness at the band point, planted sign errors in each adjoint pair, and
next to a mesh point every term has a finite limit with the corrections while
the uncorrected terms diverge).
"""
import math

import numpy as np

from . import cell as CL
from .operator import FOUR_PI, TERMS, TCOperator


def _offsets(lattice, kmesh, alpha, kcart):
    """p = k - K for every K of the Born-von Karman reciprocal lattice (K = q + G) with
    exp(-alpha p^2) above the tail of Eq. correction2's sums."""
    lattice = np.asarray(lattice, dtype=np.float64)
    kmesh = np.asarray(kmesh)
    Bs = CL.reciprocal(lattice) / kmesh[:, None]
    Ssc = lattice * kmesh[:, None]
    kcart = np.asarray(kcart, dtype=np.float64)
    pmax = np.sqrt(-np.log(CL.ALPHA_TAIL) / alpha) + np.linalg.norm(kcart)
    bound = [int(np.ceil(pmax * np.linalg.norm(Ssc[i]) / (2.0 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-b, b + 1) for b in bound]
    l = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    return kcart[None, :] - l @ Bs


def aux_scalar_sum(lattice, kmesh, alpha, kcart):
    """sum_{q,G} A_aux(k - q + G), A_aux(p) = exp(-alpha p^2)/p^2, for k off the SCF mesh."""
    p = _offsets(lattice, kmesh, alpha, kcart)
    p2 = np.einsum("ij,ij->i", p, p)
    if np.any(p2 == 0.0):
        raise ValueError("k lies on the SCF mesh")
    return math.fsum(np.exp(-alpha * p2) / p2)


def aux_vector_sum(lattice, kmesh, alpha, kcart):
    """W(k) = sum_{q,G} (k - q + G) A_aux(k - q + G) (the p = 0 term, if any, excluded)."""
    p = _offsets(lattice, kmesh, alpha, kcart)
    p2 = np.einsum("ij,ij->i", p, p)
    keep = p2 > 0.0
    t = p[keep] * (np.exp(-alpha * p2[keep]) / p2[keep])[:, None]
    return np.array([math.fsum(t[:, i]) for i in range(3)])


def gamma_band(lattice, kmesh, alpha, kcart):
    """Gamma_b(k) = Omega/(4 sqrt(pi^3 alpha)) - (1/N_k) sum_{q,G} A_aux(k - q + G)."""
    Omega = abs(float(np.linalg.det(np.asarray(lattice, dtype=np.float64))))
    Nk = int(np.prod(kmesh))
    return Omega / (4.0 * np.sqrt(np.pi ** 3 * alpha)) - aux_scalar_sum(lattice, kmesh, alpha, kcart) / Nk


class BandSetup(CL.Setup):
    """The SCF setup with band k-points appended as output-only points (indices Nk .. Nk + nkb - 1).

    Nk stays the number of mesh points, so every partner loop of the operator
    runs over the mesh alone."""

    def __init__(self, S, kfrac_band):
        self.__dict__.update(S.__dict__)
        kfb = np.atleast_2d(np.asarray(kfrac_band, dtype=np.float64))
        self.nkb = len(kfb)
        kcb = kfb @ S.B
        mb = [CL.sphere_miller(k, S.B, S.ecut) for k in kcb]
        for m in mb:
            for i in range(3):
                if np.abs(m[:, i]).max() > (S.n[i] - 1) // 2:
                    raise ValueError("band-point sphere does not fit the FFT box")
        self.on_mesh = []
        for kf in kfb:
            d = kf[None, :] - S.kfrac
            hit = np.nonzero(np.all(np.abs(d - np.round(d)) < 1e-12, axis=1))[0]
            if len(hit) and np.any(d[hit[0]] != 0.0):
                raise ValueError("a band point on the mesh must be given by the mesh point's own coordinates")
            self.on_mesh.append(int(hit[0]) if len(hit) else -1)
        self.kfrac = np.vstack([S.kfrac, kfb])
        self.kcart = np.vstack([S.kcart, kcb])
        self.miller = list(S.miller) + mb
        self.npw = np.concatenate([S.npw, np.array([len(m) for m in mb], dtype=np.int64)])
        self.npw_max = int(self.npw.max())
        self.box_index = list(S.box_index) + [tuple((m[:, i] % S.n[i]) for i in range(3)) for m in mb]
        self.gamma_b = [gamma_band(S.lattice, S.kmesh, S.alpha, kcb[i]) if self.on_mesh[i] < 0 else None
                        for i in range(self.nkb)]
        self.W = [aux_vector_sum(S.lattice, S.kmesh, S.alpha, kcb[i]) for i in range(self.nkb)]


class BandOperator(TCOperator):
    """TCOperator on a BandSetup: outputs at the band points, partners on the mesh."""

    def __init__(self, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ, left=False, backend=None):
        super().__init__(SB, c_phi, c_chi, occ, left=left, backend=backend)
        bk = self.bk
        ket_b, bra_b = (b_chi, b_phi) if self.left else (b_phi, b_chi)
        for i in range(SB.nkb):
            kb = SB.Nk + i
            self.ket.append(bk.orbital(ket_b[i], kb))
            self.bra.append(bk.orbital(bra_b[i], kb))
            self.gket.append(bk.orbital_grad(ket_b[i], kb))
        b_occ = np.asarray(b_occ, dtype=np.float64).reshape(SB.nkb, SB.nbands)
        self.f = np.vstack([self.f, b_occ[:, : SB.nocc]])   # rows Nk.. : the band points' own occupations

    def _off_mesh(self, k):
        return k >= self.S.Nk and self.S.on_mesh[k - self.S.Nk] < 0

    def _overlaps(self, k):
        """<bra_mu|ket_j> for the occupied mu and every band j at point k, shape (nocc, nbands)."""
        bk, no = self.bk, self.S.nocc
        rho = bk.mul(bk.conj(self.bra[k][:no])[:, None], self.ket[k][None])
        return bk.spec_at_zero(bk.FT(rho))

    def _corr_2ax_band(self, k):
        """Eq. divcorr_2ax_band: -(4 pi Gamma_b/Omega) sum_mu f_mu <bra_mu|ket_j> ket_mu."""
        S, bk, no = self.S, self.bk, self.S.nocc
        O = self._overlaps(k)
        c = FOUR_PI * S.gamma_b[k - S.Nk] / S.Omega
        w = self.f[k][:, None] * O                                       # (no, nb)
        return -c * np.sum(w[:, :, None, None, None] * self.ket[k][:no][:, None], axis=0)

    def _corr_3b6(self, k):
        if not self._off_mesh(k):
            return super()._corr_3b6(k)
        # Eq. 3b6_div_band1 (multiplicity 2 times 1/2, as the SCF forms)
        S, bk = self.S, self.bk
        no, Om = S.nocc, S.Omega
        O = self._overlaps(k)
        n0 = bk.spec_at_zero(self.nt)
        one = bk.const(1.0)[None]
        out = bk.zeros((S.nbands,))
        gb = S.gamma_b[k - S.Nk]
        W = S.W[k - S.Nk]
        WG = np.einsum("...i,i->...", S.Gbox, W)                              # W . G over the box
        nt = self.nt
        ntneg = bk.spec_neg(nt)
        F = bk.FT(bk.mul(bk.conj(self.bra[k][:no])[:, None], self.ket[k][None]))   # (no, nb)
        for s in range(2):
            c = (FOUR_PI * self.ks.amp(s)) ** 2 * gb
            a = FOUR_PI * self.ks.amp(s) / S.Nk
            V2 = bk.iFT(WG * self.us[s] * nt)                                  # band2 field
            X3 = np.sum(WG * self.us[s] * F * ntneg, axis=(-3, -2, -1))      # band3 scalars (no, nb)
            for q in range(no):
                field = ((c * n0) * O[q][:, None, None, None] * one                   # band1
                         - a * O[q][:, None, None, None] * V2[None]                   # band2
                         - a * X3[q][:, None, None, None] * one)                      # band3
                out = out + self.f[k][q] * bk.mul(self.ket[k][q][None], field) / (Om * Om)
        return out

    def _corr_gradu_band(self, k, acc):
        """Eqs. divcorr_2bx1/2, divcorr_3a3, div_corr_3b3_2 at an off-mesh band point (added to acc)."""
        S, bk, no = self.S, self.bk, self.S.nocc
        W = S.W[k - S.Nk]
        c = FOUR_PI * self.ks.amp(0) / (S.Nk * S.Omega)
        f = self.f[k]
        ket_m, bra_m_c = self.ket[k][:no], bk.conj(self.bra[k][:no])
        O = self._overlaps(k)                                                  # (no, nb)

        def wsum(vec_field):                                                   # W . (3, grid) -> grid
            return sum(W[d] * vec_field[..., d, :, :, :] for d in range(3))

        if "2bx1" in acc:
            Wg = wsum(self.gket[k][:no])                                       # (no, grid): W . grad ket_m
            acc["2bx1"] = acc["2bx1"] + self.s2b * 1j * c * np.sum(
                (f[:, None] * O)[:, :, None, None, None] * Wg[:, None], axis=0)
        if "2bx2" in acc:
            D = bk.spec_at_zero(bk.FT(bk.mul(bra_m_c[:, None, None], self.gket[k][None])))   # (no, nb, 3)
            WD = D @ W
            acc["2bx2"] = acc["2bx2"] - self.s2b * 1j * c * np.sum(
                (f[:, None] * WD)[:, :, None, None, None] * ket_m[:, None], axis=0)
        if "3a3" in acc:
            hW = wsum(self.h1)                                                  # grid
            t = bk.mul(hW[None], ket_m)                                         # (no, grid)
            acc["3a3"] = acc["3a3"] - 1j * c * np.sum((f[:, None] * O)[:, :, None, None, None] * t[:, None], axis=0)
        if "3b3" in acc:
            hW = wsum(self.h1)
            E = bk.spec_at_zero(bk.FT(bk.mul(bra_m_c[:, None], bk.mul(hW[None], self.ket[k])[None])))  # (no, nb)
            acc["3b3"] = acc["3b3"] + 1j * c * np.sum((f[:, None] * E)[:, :, None, None, None] * ket_m[:, None],
                                                       axis=0)
        if "3a4" in acc or "3b5" in acc:
            h3a, h3b = self._band_h3(k)
            if "3a4" in acc:     # Eqs. div_corr_3a4_2/3: + i c sum_m f_m O_mj (W . h3a(m))
                t = wsum(h3a)                                                   # (no, grid)
                acc["3a4"] = acc["3a4"] + 1j * c * np.sum((f[:, None] * O)[:, :, None, None, None] * t[:, None],
                                                           axis=0)
            if "3b5" in acc:     # Eqs. 3b5_div_2/3: - i c sum_m f_m (W . FT[ket_j h3b(m)](0)) ket_m
                E = bk.spec_at_zero(bk.FT(bk.mul(self.ket[k][None, :, None], h3b[:, None])))   # (no, nb, 3)
                acc["3b5"] = acc["3b5"] - 1j * c * np.sum((f[:, None] * (E @ W))[:, :, None, None, None]
                                                          * ket_m[:, None], axis=0)
        if "3b4" in acc:         # Eqs. div_corr_3b4_2 (on w_j) and div_corr_3b4_4
            wc = -1j * c * np.einsum("d,mj,m...->jd...", W, f[:, None] * O, ket_m)      # correction of w_j
            w = self._w_last + wc
            acc["3b4"] = acc["3b4"] - self._pass_3b4(k, wc)
            E = bk.spec_at_zero(bk.FT(bk.mul(bra_m_c[:, None, None], w[None])))          # (no, nb, 3)
            acc["3b4"] = acc["3b4"] - 1j * c * np.sum((f[:, None] * (E @ W))[:, :, None, None, None]
                                                      * ket_m[:, None], axis=0)
        return acc

    def _band_h3(self, k):
        """h3 of both kinds for the band point's own occupied orbitals m (q2 at k_b, partners q1 on the
        mesh; Algs. 6 and 8 with kernels at k_b - q1 + G and q1 - k_b + G), each with the correction of
        Eq. correction_nabla for q1 -> k_b (the source of Eqs. div_corr_3a4_3 and 3b5_div_3):
          h3a(m) = sum_q1 f/N_k P(q1, m) ket_q1   - i c W sum_m' f_m' <bra_m'|ket_m> ket_m'
          h3b(m) = sum_q1 f/N_k P(m, q1) bra_q1^* + i c W sum_m' f_m' <bra_m|ket_m'> bra_m'^*
        Returns (h3a, h3b), each (nocc, 3, grid)."""
        S, bk = self.S, self.bk
        Nk, no = S.Nk, S.nocc
        c = FOUR_PI * self.ks.amp(0) / (Nk * S.Omega)
        W = S.W[k - Nk]
        ket_m, bra_m_c = self.ket[k][:no], bk.conj(self.bra[k][:no])
        h3a = bk.zeros((no, 3))
        h3b = bk.zeros((no, 3))
        for k1 in range(Nk):
            f1 = self.f[k1] / Nk
            bra1_c, ket1 = bk.conj(self.bra[k1][:no]), self.ket[k1][:no]
            KB = self.kern(k, k1)                                                   # p = k_b - q1 + G
            PB = bk.iFT(KB["U"][0][None, None] * bk.FT(bk.mul(bra1_c[:, None], ket_m[None]))[:, :, None])
            h3a = h3a + np.sum(f1[:, None, None, None, None, None] * bk.mul(PB, ket1[:, None, None]), axis=0)
            KA = self.kern(k1, k)                                                   # p = q1 - k_b + G
            PA = bk.iFT(KA["U"][0][None, None] * bk.FT(bk.mul(bra_m_c[:, None], ket1[None]))[:, :, None])
            h3b = h3b + np.sum(f1[None, :, None, None, None, None] * bk.mul(PA, bra1_c[None, :, None]), axis=1)
        Ob = self._overlaps(k)[:, :no]                                             # [m', m] = <bra_m'|ket_m>
        f = self.f[k]
        h3a = h3a - 1j * c * np.einsum("d,pm,p...->md...", W, f[:, None] * Ob, ket_m)
        h3b = h3b + 1j * c * np.einsum("d,mp,p...->md...", W, Ob * f[None, :], bra_m_c)
        return h3a, h3b

    def apply_band(self, terms=TERMS):
        """Per-term outputs {term: (nkb, nbands, npw_max)} at the band points."""
        self.prepare()
        S = self.S
        res = {t: np.zeros((S.nkb, S.nbands, S.npw_max), dtype=np.complex128) for t in terms}
        for i in range(S.nkb):
            kb = S.Nk + i
            acc = self._apply_k(kb, terms)
            if S.div_correction and self._off_mesh(kb):
                if "2ax" in acc:
                    acc["2ax"] = acc["2ax"] + self._corr_2ax_band(kb)
                acc = self._corr_gradu_band(kb, acc)
            for t in terms:
                res[t][i] = self.bk.project(acc[t], kb)
        return res


def _pad(c, npw_max):
    c = np.asarray(c, dtype=np.complex128)
    out = np.zeros(c.shape[:-1] + (npw_max,), dtype=np.complex128)
    out[..., : c.shape[-1]] = c
    return out


def band_apply(S, c_phi, c_chi, occ, kfrac_band, b_phi, b_chi, b_occ, left=False, terms=TERMS, backend=None):
    """Right (left=True: left) operator on the orbitals of the band points kfrac_band.

    c_phi, c_chi, occ: the SCF mesh orbitals and occupations (the partners);
    b_phi, b_chi: (nkb, nbands, npw) band-point orbitals on the spheres of
    ``BandSetup(S, kfrac_band)``; b_occ: (nkb, nbands) their occupations (the
    first nocc are the band point's own occupied orbitals).  Returns
    {term: (nkb, nbands, npw_max)} on those spheres.
    """
    SB = BandSetup(S, kfrac_band)
    n = SB.npw_max
    op = BandOperator(SB, _pad(c_phi, n), _pad(c_chi, n), occ, _pad(b_phi, n), _pad(b_chi, n), b_occ,
                      left=left, backend=backend(SB) if backend else None)
    return op.apply_band(terms=terms)
