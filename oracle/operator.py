"""The TC / BITC two- and three-body operator and the TC pseudo-energy (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 2.6 of arXiv:2302.07420 step by step.  One spin channel is
computed (non-spin-polarised, the two spin channels hold identical orbitals):
exchange-type terms pair same-spin orbitals only and use the parallel-spin
Jastrow (A_pp, C_pp); Hartree-type sums and the sums over a free spin index in
3a2 and 3b6 take both channels, i.e. pp + ap kernels.

Units.  An orbital is held as psi(r) = sum_G c(G) e^{iG.r} = sqrt(Omega)
phi_periodic(r) (the dimensionless array of Sec. 2.6.1), with sum |c|^2 = 1.
Every kernel K of the paper then enters divided by Omega (K^ = K/Omega), the
density is n_psi = (1/N_k) sum_q f_q chi_q^* phi_q in the same units, and the
output coefficients are those of g_j in the units of c.

Right operator, for an output orbital j at k (ket x = phi_j), with
rho_qj = chi_q^* phi_j, Delta = k - q, U^_s(p) = i p u~_s(p)/Omega (zero at p = 0)
and P^s(a, b) = FT^{-1}[U^_s(k_b - k_a + G) FT[chi_a^* phi_b]]:

  2ah   Alg. 1        v_H phi_j,          v_H = FT^{-1}[(V^pp + V^ap)^ n~]  (G != 0)
  2bh1  Sec. 2.6.3    h1 . grad phi_j,    h1 = FT^{-1}[i G (u~pp + u~ap)^ n~]
  2bh2  Sec. 2.6.3    v_b2 phi_j,         v_b2 = FT^{-1}[-i G (u~pp + u~ap)^ . m~],
                                          m = (1/N_k) sum_q f_q chi_q^* grad phi_q
  2ax   Alg. 2        -sum_q f_q/N_k phi_q FT^{-1}[V^pp(Delta + G) rho~_qj]
  2bx1  Sec. 2.6.3    -sum_q f_q/N_k grad phi_q . FT^{-1}[U^pp rho~_qj]
  2bx2  Sec. 2.6.3    +sum_q f_q/N_k phi_q FT^{-1}[U^pp . FT[chi_q^* grad phi_j]]
  3a1   Alg. 3        -(1/2) (h1 . h1) phi_j
  3a2   Alg. 4        (1/2) h6 phi_j,     h6 = sum_{q1,q2} f f/N_k^2 sum_s P^s(q2,q1) . P^s(q1,q2)
  3a3   Alg. 5        (1/2) h1 . w_j,     w_j = sum_q f_q/N_k phi_q FT^{-1}[U^pp rho~_qj]
  3a4   Alg. 6        -(1/2) sum_q2 f/N_k h3(q2) . FT^{-1}[U^pp(k - q2 + G) rho~_q2j],
                                          h3(q2) = sum_q1 f/N_k P^pp(q1,q2) phi_q1
  3b1   Alg. 7        -(1/2) FT^{-1}[-i G u~^ . FT[h1 n]] phi_j
  3b2   Alg. 8        (1/2) FT^{-1}[-i G u~^ . FT[h5]] phi_j,  h5 = sum_q2 f/N_k h3b(q2) phi_q2,
                                          h3b(q2) = sum_q1 f/N_k P^pp(q2,q1) chi_q1^*
  3b3   Alg. 9        (1/2) sum_q f/N_k phi_q FT^{-1}[-U^pp . FT[h1 rho_qj]]
  3b4   Alg. 10       -(1/2) sum_q f/N_k phi_q FT^{-1}[-U^pp . FT[chi_q^* w_j]]
                      (the accumulation of h3 is read as h3 += h2 phi_q2, the
                      printed "h3 += h3 phi" being a typo; h3 then equals w_j)
  3b5   Alg. 11       -(1/2) sum_q2 f/N_k phi_q2 FT^{-1}[-U^pp . FT[phi_j h3b(q2)]]
  3b6   Alg. 12       (1/2) sum_q2 f/N_k phi_q2 FT^{-1}[sum_s -U^s . FT[n FT^{-1}[U^s rho~_q2j]]]

Multiplicities (Sec. 2.6.4): the full three-body operator is
3a1 + 3a2 + 2*3a3 + 2*3a4 + 2*(3b1 + ... + 3b6) because 3a5 = 3a4, 3a6 = 3a3 and
3c* = 3b*; the outputs below carry these factors.  The printed |h1|^2 of
Algorithm 3 is read as h1 . h1 (no conjugate): the integrand has two bra
densities chi^* phi, which are complex for BITC; for TC h1 is real and the two agree.

Left operator (Eq. BITCSCFconj): the same algorithms with phi <-> chi, the
V_2a kernel replaced by V_2a^dagger and the signs of the four grad u . grad
terms (2bh1, 2bh2, 2bx1, 2bx2) flipped.  With V_2a^dagger(0) = V_2a(0) (see
``kernels.V2a_jastrow_zero``) this is exactly the adjoint of the discrete right
operator, so <chi_i|h phi_j> = <h^dagger chi_i|phi_j>.

Divergence corrections for k on the SCF mesh, with
Gamma0 = Omega/(4 sqrt(pi^3 alpha)) - (1/N_k)(-alpha + sum' A_aux) (Eq. correction2):
  2ax   Eq. divcorr_2ax_scf: the Coulomb 4 pi/p^2 at p = 0 is replaced by 4 pi N_k Gamma0,
        i.e. -4 pi Gamma0 sum_mu f <chi_qk|phi_j>/Omega phi_qk; the Jastrow parts of V_2a keep
        their finite p = 0 values.
  3a2   Eqs. divcor_3a2_first/second in their general-overlap form (Eqs. ..._density_matrix_mixing),
        added to h5(q2):  [(4 pi A)^2 Gamma0 + x 4 pi A u_short/N_k] F0 / Omega^2
        + (4 pi A/N_k)/Omega^2 sum_{G != 0} u~(G) (F_a(G) + F_b(G)) e^{iG.r}, x = ushort_factor.
  3b6   Eqs. 3b6_div_scf1/2/3 (times the multiplicity 2).
The grad-u (odd) corrections of 2bx1, 2bx2, 3a3, 3a4, 3b3, 3b4, 3b5 vanish for
k on the uniform SCF mesh (Sec. 2.5, Eq. correction_nabla) and are not added.

Energy (Eqs. EtotTC / EtotBiTC, single determinant): per unit cell, both spins,
E = (2/N_k) Re sum_{k,mu} f [<chi|T|phi> + (1/2) <chi|g_2> + (1/3) <chi|g_3>].

Parity pins: tests/test_oracle_*.py (direct-sum backend, HEG closed forms, HF
limit, gauge, adjointness, translation, quadratic in A, energy gradient).
"""
import numpy as np

from . import kernels as KN
from .backends import FFTBackend

TWO_BODY = ("2ah", "2bh1", "2bh2", "2ax", "2bx1", "2bx2")
THREE_BODY = ("3a1", "3a2", "3a3", "3a4", "3b1", "3b2", "3b3", "3b4", "3b5", "3b6")
TERMS = TWO_BODY + THREE_BODY
FOUR_PI = 4.0 * np.pi


class TCOperator:
    """Right (left=False) or left (left=True) TC operator for fixed orbitals."""

    def __init__(self, S, c_phi, c_chi, occ, left=False, backend=None, kset=None, sym=None):
        self.S = S
        # symmetry-reduced occupied-pair stage: (ops, kinfo, irred) of oracle.symmetry, or None
        self.sym = sym
        self.bk = backend if backend is not None else FFTBackend(S)
        # Jastrow kernel data (values at S.A, S.C unless a displaced set is given, see gradient.py)
        self.ks = kset if kset is not None else KN.JastrowKernels(S.A, S.C)
        self.left = bool(left)
        self.s2b = -1.0 if self.left else 1.0
        c_phi = np.asarray(c_phi, dtype=np.complex128)
        c_chi = np.asarray(c_chi, dtype=np.complex128)
        ket_c, bra_c = (c_chi, c_phi) if self.left else (c_phi, c_chi)
        self.occ = np.asarray(occ, dtype=np.float64).reshape(S.Nk, S.nbands)
        self.f = self.occ[:, : S.nocc]
        bk = self.bk
        self.ket = [bk.orbital(ket_c[k], k) for k in range(S.Nk)]        # (nb, grid)
        self.bra = [bk.orbital(bra_c[k], k) for k in range(S.Nk)]
        self.gket = [bk.orbital_grad(ket_c[k], k) for k in range(S.Nk)]  # (nb, 3, grid)
        self._kcache = {}
        self._prepared = False

    # ------------------------------------------------------------------ kernels
    def kern(self, kout, kpart):
        """Kernel spectra at p = k_out - k_part + G over the FFT box (divided by Omega)."""
        key = (kout, kpart)
        if key in self._kcache:
            return self._kcache[key]
        S = self.S
        delta = S.kcart[kout] - S.kcart[kpart]
        p = delta[None, None, None, :] + S.Gbox
        p2 = np.einsum("...i,...i->...", p, p)
        zero = p2 == 0.0
        p2s = np.where(zero, 1.0, p2)
        ks = self.ks
        V = ks.V2a(p2s, 0, adjoint=self.left)
        v0 = ks.v0(0)
        if S.div_correction:
            v0 = v0 + ks.coulomb_zero(S.Nk, S.Gamma0)
        V = np.where(zero, v0, V) / S.Omega
        U = []
        for s in range(2):
            u = np.where(zero, 0.0, ks.u(p2s, s)) / S.Omega
            U.append(1j * np.moveaxis(p, -1, 0) * u[None])              # (3, grid)
        out = {"V": V, "U": U}
        self._kcache[key] = out
        return out

    def hartree_kernels(self):
        S = self.S
        G = S.Gbox
        g2 = np.einsum("...i,...i->...", G, G)
        zero = g2 == 0.0
        g2s = np.where(zero, 1.0, g2)
        ks = self.ks
        Vh = sum(ks.V2a(g2s, s, adjoint=self.left) for s in range(2))
        uh = sum(ks.u(g2s, s) for s in range(2))
        Vh = np.where(zero, 0.0, Vh) / S.Omega
        uh = np.where(zero, 0.0, uh) / S.Omega
        Uh = 1j * np.moveaxis(G, -1, 0) * uh[None]
        us = [np.where(zero, 0.0, ks.u(g2s, s)) for s in range(2)]  # no 1/Omega
        return Vh, Uh, us

    # ------------------------------------------------------------------ stages
    def prepare(self):
        """Densities, Hartree-type fields and the occupied-pair stage (Algs. 4, 6, 8, 11)."""
        if self._prepared:
            return
        S, bk = self.S, self.bk
        Nk, no = S.Nk, S.nocc
        # spin density (per spin) and the vector density of 2bh2
        n = bk.zeros()
        m = bk.zeros((3,))
        for k in range(Nk):
            cb = bk.conj(self.bra[k][:no])
            w = self.f[k][:, None, None, None] / Nk
            n = n + np.sum(w * bk.mul(cb, self.ket[k][:no]), axis=0)
            m = m + np.sum(w[:, None] * bk.mul(cb[:, None], self.gket[k][:no]), axis=0)
        self.n, self.m = n, m
        Vh, Uh, us = self.hartree_kernels()
        self.Uh, self.us = Uh, us
        nt = bk.FT(n)
        self.nt = nt
        self.vH = bk.iFT(Vh * nt)                                     # Alg. 1
        self.h1 = bk.iFT(Uh * nt[None])                               # Alg. 3 (h1)
        mt = bk.FT(m)
        self.vb2 = bk.iFT(np.sum(-Uh * mt, axis=0))
        h1n = bk.FT(bk.mul(self.h1, n[None]))                         # Alg. 7
        self.t3b1 = bk.iFT(np.sum(-Uh * h1n, axis=0))
        self._occupied_pairs()
        self._prepared = True

    def _occupied_pairs(self):
        S, bk = self.S, self.bk
        Nk, no = S.Nk, S.nocc
        h6 = bk.zeros()
        h3a4 = [bk.zeros((no, 3)) for _ in range(Nk)]
        h3b = [bk.zeros((no, 3)) for _ in range(Nk)]
        c6 = [bk.zeros() for _ in range(Nk)]              # h6 contribution of each q2's k-point
        k2_list = range(Nk) if self.sym is None else self.sym[2]
        for k2 in k2_list:
            for k1 in range(Nk):
                # rhoA[q2, q1] = chi_q2^* phi_q1 (kernel at k1 - k2); rhoB[q1, q2] = chi_q1^* phi_q2
                rhoA = bk.mul(bk.conj(self.bra[k2][:no])[:, None], self.ket[k1][:no][None])
                rhoB = bk.mul(bk.conj(self.bra[k1][:no])[:, None], self.ket[k2][:no][None])
                FA = bk.FT(rhoA)
                FB = bk.FT(rhoB)
                KA = self.kern(k1, k2)
                KB = self.kern(k2, k1)
                w = (self.f[k2][:, None] * self.f[k1][None, :]) / (Nk * Nk)   # [q2, q1]
                for s in range(2):
                    PA = bk.iFT(KA["U"][s][None, None] * FA[:, :, None])   # P^s(q2,q1)  (no2, no1, 3)
                    PB = bk.iFT(KB["U"][s][None, None] * FB[:, :, None])   # P^s(q1,q2)  (no1, no2, 3)
                    prod = np.sum(bk.mul(PA, np.swapaxes(PB, 0, 1)), axis=2)  # (no2, no1)
                    c6[k2] = c6[k2] + np.sum(w[:, :, None, None, None] * prod, axis=(0, 1))
                    if s == 0:
                        f1 = self.f[k1] / Nk
                        # h3(q2) += f1 P^pp(q1,q2) phi_q1            (Alg. 6)
                        t = bk.mul(PB, self.ket[k1][:no][:, None, None])
                        h3a4[k2] = h3a4[k2] + np.sum(f1[:, None, None, None, None, None] * t, axis=0)
                        # h3b(q2) += f1 P^pp(q2,q1) chi_q1^*         (Alg. 8)
                        t = bk.mul(PA, bk.conj(self.bra[k1][:no])[None, :, None])
                        h3b[k2] = h3b[k2] + np.sum(f1[None, :, None, None, None, None] * t, axis=1)
        if S.div_correction:
            for k2 in k2_list:
                c6[k2] = c6[k2] + self._corr_3a2(k2)
        if self.sym is not None:
            # Sec. 2.6.4: fields of q2 from those of its irreducible q2;0
            from . import symmetry as SY
            ops, kinfo, _ = self.sym
            for k2 in range(Nk):
                k0, op, tr, K = kinfo[k2]
                if k2 == k0:
                    continue
                h3a4[k2] = SY.rotate_field(S, h3a4[k0], ops[op], tr, K, vector=True)
                h3b[k2] = SY.rotate_field(S, h3b[k0], ops[op], tr, -K, vector=True)
                c6[k2] = SY.rotate_field(S, c6[k0], ops[op], tr, 0 * K, vector=False)
        for k2 in range(Nk):
            h6 = h6 + c6[k2]
        self.h6 = h6
        self.h3a4 = h3a4
        self.h3b = h3b
        # h5 of Alg. 8 and the 3b2 potential
        h5 = bk.zeros((3,))
        for k in range(Nk):
            t = bk.mul(h3b[k], self.ket[k][:no][:, None])
            h5 = h5 + np.sum((self.f[k] / Nk)[:, None, None, None, None] * t, axis=0)
        self.h5 = h5
        self.t3b2 = bk.iFT(np.sum(-self.Uh * bk.FT(h5), axis=0))

    def _corr_3a2(self, k):
        """Eqs. divcor_3a2_first/second (general-overlap form) of the q2 at k-point k, added to h6."""
        S, bk = self.S, self.bk
        Nk, no, Om = S.Nk, S.nocc, S.Omega
        out = bk.zeros()
        rho = bk.mul(bk.conj(self.bra[k][:no])[:, None], self.ket[k][:no][None])  # [a, b] = chi_a^* phi_b
        F = bk.FT(rho)
        O = bk.spec_at_zero(F)                                                      # <chi_a|phi_b>
        f = self.f[k]
        for q2 in range(no):
            F0 = np.sum(f * O[q2, :] * O[:, q2])
            Fa = np.sum((f * O[:, q2])[:, None, None, None] * F[q2, :], axis=0)  # FT[chi_q2^* phi_q1](G) <chi_q1|phi_q2>
            Fb = np.sum((f * O[q2, :])[:, None, None, None] * F[:, q2], axis=0)  # <chi_q2|phi_q1> FT[chi_q1^* phi_q2](G)
            for s in range(2):
                c = self.ks.corr(s, S.Gamma0, S.ushort_factor, Nk)
                field = bk.const(c * F0) + (FOUR_PI * self.ks.amp(s) / Nk) * bk.iFT(self.us[s] * (Fa + Fb))
                out = out + (f[q2] / Nk) * field / (Om * Om)
        return out

    # ------------------------------------------------------------------ apply
    def apply(self, kpoints=None, terms=TERMS):
        """Per-term outputs {term: (Nk, nb, npw_max)} for the requested output k-points."""
        self.prepare()
        S = self.S
        kpoints = range(S.Nk) if kpoints is None else kpoints
        res = {t: np.zeros((S.Nk, S.nbands, S.npw_max), dtype=np.complex128) for t in terms}
        for k in kpoints:
            acc = self._apply_k(k, terms)
            for t in terms:
                res[t][k] = self.bk.project(acc[t], k)
        return res

    def _apply_k(self, k, terms):
        S, bk = self.S, self.bk
        Nk, no, nb = S.Nk, S.nocc, S.nbands
        s2b = self.s2b
        ketj, gketj = self.ket[k], self.gket[k]
        acc = {t: bk.zeros((nb,)) for t in terms}
        w = bk.zeros((nb, 3))

        def fsum(fq, x):
            return np.sum(fq.reshape((-1,) + (1,) * (x.ndim - 1)) * x, axis=0)

        for kq in range(Nk):
            K = self.kern(k, kq)
            braq_c = bk.conj(self.bra[kq][:no])
            ketq, gketq = self.ket[kq][:no], self.gket[kq][:no]
            fq = self.f[kq] / Nk
            rho = bk.mul(braq_c[:, None], ketj[None])                          # (no, nb)
            Fr = bk.FT(rho)
            h2V = bk.iFT(K["V"] * Fr)
            h2U = [bk.iFT(K["U"][s][None, None] * Fr[:, :, None]) for s in range(2)]  # (no, nb, 3)
            if "2ax" in acc:
                acc["2ax"] -= fsum(fq, bk.mul(ketq[:, None], h2V))
            if "2bx1" in acc:
                acc["2bx1"] -= s2b * fsum(fq, np.sum(bk.mul(gketq[:, None], h2U[0]), axis=2))
            w = w + fsum(fq, bk.mul(ketq[:, None, None], h2U[0]))
            if "3a4" in acc:   # multiplicity 2 times -(1/2)
                acc["3a4"] -= fsum(fq, np.sum(bk.mul(self.h3a4[kq][:, None], h2U[0]), axis=2))
            if "2bx2" in acc:
                X = bk.FT(bk.mul(braq_c[:, None, None], gketj[None]))           # FT[chi_q^* d phi_j]
                Y = bk.iFT(np.sum(K["U"][0][None, None] * X, axis=2))
                acc["2bx2"] += s2b * fsum(fq, bk.mul(ketq[:, None], Y))
            if "3b3" in acc:   # 2 * (1/2)
                X = bk.FT(bk.mul(self.h1[None, None], rho[:, :, None]))
                Y = bk.iFT(np.sum(-K["U"][0][None, None] * X, axis=2))
                acc["3b3"] += fsum(fq, bk.mul(ketq[:, None], Y))
            if "3b5" in acc:   # 2 * (-1/2)
                X = bk.FT(bk.mul(ketj[None, :, None], self.h3b[kq][:, None]))
                Y = bk.iFT(np.sum(-K["U"][0][None, None] * X, axis=2))
                acc["3b5"] -= fsum(fq, bk.mul(ketq[:, None], Y))
            if "3b6" in acc:   # 2 * (1/2)
                Ysum = 0.0
                for s in range(2):
                    X = bk.FT(bk.mul(self.n[None, None, None], h2U[s]))
                    Ysum = Ysum + np.sum(-K["U"][s][None, None] * X, axis=2)
                acc["3b6"] += fsum(fq, bk.mul(ketq[:, None], bk.iFT(Ysum)))
        self._w_last = w       # w_j of this k-point (read by the band-point corrections)
        if "3b4" in acc:       # second pass: w_j is complete; 2 * (-1/2)
            acc["3b4"] -= self._pass_3b4(k, w)
        # Hartree-type (local) terms
        if "2ah" in acc:
            acc["2ah"] += bk.mul(self.vH[None], ketj)
        if "2bh1" in acc:
            acc["2bh1"] += s2b * np.sum(bk.mul(self.h1[None], gketj), axis=1)
        if "2bh2" in acc:
            acc["2bh2"] += s2b * bk.mul(self.vb2[None], ketj)
        if "3a1" in acc:
            acc["3a1"] += -0.5 * bk.mul(np.sum(bk.mul(self.h1, self.h1), axis=0)[None], ketj)
        if "3a2" in acc:
            acc["3a2"] += 0.5 * bk.mul(self.h6[None], ketj)
        if "3a3" in acc:   # 2 * (1/2)
            acc["3a3"] += np.sum(bk.mul(self.h1[None], w), axis=1)
        if "3b1" in acc:   # 2 * (-1/2)
            acc["3b1"] += -bk.mul(self.t3b1[None], ketj)
        if "3b2" in acc:   # 2 * (1/2)
            acc["3b2"] += bk.mul(self.t3b2[None], ketj)
        if "3b6" in acc and S.div_correction:
            acc["3b6"] += self._corr_3b6(k)
        return acc

    def _pass_3b4(self, k, w):
        """Alg. 10 for the orbitals of k-point k given w (nb, 3, grid): sum_q f/N_k ket_q FT^{-1}[-U . FT[bra_q^* w]]."""
        S, bk = self.S, self.bk
        Nk, no = S.Nk, S.nocc
        out = 0.0
        for kq in range(Nk):
            K = self.kern(k, kq)
            braq_c = bk.conj(self.bra[kq][:no])
            X = bk.FT(bk.mul(braq_c[:, None, None], w[None]))
            Y = bk.iFT(np.sum(-K["U"][0][None, None] * X, axis=2))
            fq = self.f[kq] / Nk
            out = out + np.sum(fq.reshape((-1,) + (1,) * (Y.ndim - 1)) * bk.mul(self.ket[kq][:no][:, None], Y), axis=0)
        return out

    def _corr_3b6(self, k):
        """Eqs. 3b6_div_scf1/2/3 (times the multiplicity 2 of 3b*, times 1/2 of 3b6)."""
        S, bk = self.S, self.bk
        Nk, no, Om = S.Nk, S.nocc, S.Omega
        rho = bk.mul(bk.conj(self.bra[k][:no])[:, None], self.ket[k][None])   # (no, nb)
        F = bk.FT(rho)
        O = bk.spec_at_zero(F)                                                 # (no, nb)
        nt = self.nt
        n0 = bk.spec_at_zero(nt)
        ntneg = bk.spec_neg(nt)
        out = bk.zeros((S.nbands,))
        for s in range(2):
            c = self.ks.corr(s, S.Gamma0, S.ushort_factor, Nk)
            A = self.ks.amp(s)
            vu = bk.iFT(self.us[s] * nt)                                          # sum_{G!=0} u~(G) n~(G) e^{iG.r}
            X = np.sum(self.us[s] * F * ntneg, axis=(-3, -2, -1))               # (no, nb)
            one = bk.const(1.0)[None]
            for q in range(no):
                field = ((c * n0) * O[q][:, None, None, None] * one                     # scf1
                         + (FOUR_PI * A / Nk) * O[q][:, None, None, None] * vu[None]    # scf2
                         + (FOUR_PI * A / Nk) * X[q][:, None, None, None] * one)        # scf3
                out = out + self.f[k][q] * bk.mul(self.ket[k][q][None], field) / (Om * Om)
        return out


def apply_operator(S, c_phi, c_chi, occ, left=False, kpoints=None, terms=TERMS, backend=None, kset=None, sym=None):
    op = TCOperator(S, c_phi, c_chi, occ, left=left, backend=backend(S) if backend else None, kset=kset, sym=sym)
    return op.apply(kpoints=kpoints, terms=terms)


def total(res, terms=None):
    terms = terms if terms is not None else list(res.keys())
    return sum(res[t] for t in terms)


def tc_apply(S, c_phi, c_chi, occ, kpoints=None, backend=None):
    """(out_R, out_L): two- plus three-body operator applied to every right / left orbital."""
    r = apply_operator(S, c_phi, c_chi, occ, left=False, kpoints=kpoints, backend=backend)
    l = apply_operator(S, c_phi, c_chi, occ, left=True, kpoints=kpoints, backend=backend)
    return total(r), total(l)


def kinetic_coeffs(S, c):
    """T c = |k+G|^2/2 c on every sphere (Sec. 2.6.2)."""
    out = np.zeros_like(c)
    for k in range(S.Nk):
        kg = S.kpG(k)
        out[k, :, : S.npw[k]] = 0.5 * np.einsum("ij,ij->i", kg, kg)[None] * c[k, :, : S.npw[k]]
    return out


def energy_terms(S, c_phi, c_chi, occ, res=None, backend=None, kset=None):
    """Per-term pseudo-energies per unit cell (both spins) and their total."""
    c_phi = np.asarray(c_phi, dtype=np.complex128)
    c_chi = np.asarray(c_chi, dtype=np.complex128)
    occ = np.asarray(occ, dtype=np.float64).reshape(S.Nk, S.nbands)
    if res is None:
        res = apply_operator(S, c_phi, c_chi, occ, left=False, backend=backend, kset=kset)
    pref = 2.0 / S.Nk
    E = {}
    tk = kinetic_coeffs(S, c_phi)
    E["kin"] = pref * float(np.real(np.sum(occ[:, :, None] * np.conj(c_chi) * tk)))
    for t, v in res.items():
        wgt = 0.5 if t in TWO_BODY else 1.0 / 3.0
        E[t] = pref * wgt * float(np.real(np.sum(occ[:, :, None] * np.conj(c_chi) * v)))
    E["total"] = sum(v for kk, v in E.items())
    return E
