"""torch.autograd.Function for the TC pseudo-energy E(phi_R, phi_L, A, C).

forward runs tc_energy; backward runs tc_energy_grad.  Only the orbitals are
saved between the two: every pair density is recomputed in the backward pass.
The orbital gradients are the left/right operator outputs plus the kinetic
term; dE/dA and dE/dC are exact symmetric differences of the energy along the
derivative of the kernel data (the energy is quadratic in that data).

Complex gradients follow PyTorch's convention for real-valued functions:
grad = dE/dRe(c) + i dE/dIm(c).

    model = TCEnergyModel(lattice, kmesh, ecut, fft, nbands, nocc)
    E = model.energy(phi_R, phi_L, A, C, occ)    # A, C: float64 tensors [pp, ap]
    E.backward()
"""
import numpy as np
import torch

from .operator import Context


class TCEnergyModel:
    """Cell, basis and precision of the energy; keeps one library context for the current (A, C)."""

    def __init__(self, lattice, kmesh, ecut, fft, nbands, nocc, alpha=0.0, div_correction=1, ushort_factor=1.0,
                 precision="fp64"):
        self.kw = dict(lattice=lattice, kmesh=kmesh, ecut=ecut, fft=fft, nbands=nbands, nocc=nocc, alpha=alpha,
                       div_correction=div_correction, ushort_factor=ushort_factor, precision=precision)
        self._ctx = None
        self._key = None

    def context(self, A, C):
        key = (tuple(float(x) for x in np.asarray(A).ravel()), tuple(float(x) for x in np.asarray(C).ravel()))
        if key != self._key:
            if self._ctx is not None:
                self._ctx.close()
            self._ctx = Context(A=list(key[0]), C=list(key[1]), **self.kw)
            self._key = key
        return self._ctx

    def energy(self, phi_R, phi_L, A, C, occ):
        return TCEnergy.apply(phi_R, phi_L, A, C, self, np.asarray(occ, dtype=np.float64))

    def close(self):
        if self._ctx is not None:
            self._ctx.close()
            self._ctx = None
            self._key = None


class TCEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi_R, phi_L, A, C, model, occ):
        Av = A.detach().cpu().numpy()
        Cv = C.detach().cpu().numpy()
        E = model.context(Av, Cv).energy(phi_R.detach(), phi_L.detach(), occ)
        ctx.save_for_backward(phi_R, phi_L)
        ctx.model, ctx.occ, ctx.AC = model, occ, (Av, Cv)
        return torch.tensor(E, dtype=torch.float64, device=A.device)

    @staticmethod
    def backward(ctx, gE):
        phi_R, phi_L = ctx.saved_tensors
        need = ctx.needs_input_grad
        orb, par = need[0] or need[1], need[2] or need[3]
        tc = ctx.model.context(*ctx.AC)
        g_phi, g_chi, dA, dC = tc.energy_grad(phi_R.detach(), phi_L.detach(), ctx.occ, orbitals=orb, params=par)
        s = gE.detach()
        out = [None] * 6
        if need[0]:
            out[0] = s.to(g_phi.device) * g_phi
        if need[1]:
            out[1] = s.to(g_chi.device) * g_chi
        if need[2]:
            out[2] = s.cpu() * torch.from_numpy(dA).to(s.dtype)
            out[2] = out[2].to(gE.device)
        if need[3]:
            out[3] = (s.cpu() * torch.from_numpy(dC).to(s.dtype)).to(gE.device)
        return tuple(out)
