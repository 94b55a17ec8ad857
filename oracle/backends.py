"""Grid algebra used by ``oracle.operator`` (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The algorithms of the paper are written with four grid operations: the
periodic transform FT (1/N normalised, Sec. 2.2), its inverse FT^{-1}, the
pointwise product of two cell-periodic functions and complex conjugation.
``FFTBackend`` stores a field by its values on the real-space grid and uses
pocketfft (scipy.fft) for FT; ``DirectBackend`` stores a field by its Fourier
coefficients on the FFT box, so FT is the identity and a pointwise product is
the cyclic convolution C(m) = sum_m' A(m') B(m - m' mod n), summed term by
term.  Running ``operator`` with both and comparing is the brute-force pin of
the FFT route (no FFT anywhere in the direct route).

Leading axes of a field are batch axes; the last three are the grid.
"""
import os

import numpy as np
import scipy.fft as sfft

_WORKERS = int(os.environ.get("TC_ORACLE_THREADS", "0")) or (os.cpu_count() or 1)


class FFTBackend:
    name = "fft"

    def __init__(self, S):
        self.S = S
        self.n = S.n
        self.N = S.N

    # --- transforms -------------------------------------------------------
    def FT(self, f):
        return sfft.fftn(f, axes=(-3, -2, -1), workers=_WORKERS) / self.N

    def iFT(self, F):
        return sfft.ifftn(F, axes=(-3, -2, -1), workers=_WORKERS) * self.N

    # --- field algebra ------------------------------------------------------
    def mul(self, a, b):
        return a * b

    def conj(self, a):
        return np.conj(a)

    def const(self, value):
        return np.full(self.n, value, dtype=np.complex128)

    def zeros(self, batch=()):
        return np.zeros(tuple(batch) + self.n, dtype=np.complex128)

    # --- orbitals -------------------------------------------------------------
    def box(self, c, k):
        """Sphere coefficients (..., npw) -> box spectrum (..., n1, n2, n3)."""
        npw = self.S.npw[k]
        out = np.zeros(c.shape[:-1] + self.n, dtype=np.complex128)
        i0, i1, i2 = self.S.box_index[k]
        out[..., i0, i1, i2] = c[..., :npw]
        return out

    def orbital(self, c, k):
        return self.iFT(self.box(c, k))

    def orbital_grad(self, c, k):
        kg = self.S.kpG(k)                                   # (npw, 3)
        npw = self.S.npw[k]
        g = 1j * c[..., None, :npw] * kg.T[None] if c.ndim == 2 else 1j * c[None, :npw] * kg.T
        return self.iFT(self.box(g, k))

    def project(self, f, k):
        """Field -> Fourier coefficients on the sphere of k (padded to npw_max)."""
        F = self.FT(f)
        i0, i1, i2 = self.S.box_index[k]
        out = np.zeros(F.shape[:-3] + (self.S.npw_max,), dtype=np.complex128)
        out[..., : self.S.npw[k]] = F[..., i0, i1, i2]
        return out

    def spec_at_zero(self, F):
        return F[..., 0, 0, 0]

    def spec_neg(self, F):
        """F(-G) on the box (index m -> -m mod n)."""
        return np.roll(np.flip(F, axis=(-3, -2, -1)), shift=1, axis=(-3, -2, -1))


class DirectBackend(FFTBackend):
    """Fields held as box spectra; FT is the identity, products are cyclic sums."""

    name = "direct"

    def __init__(self, S):
        super().__init__(S)
        n1, n2, n3 = self.n
        idx = np.arange(self.N).reshape(self.n)
        self._shift = []
        for a in range(n1):
            for b in range(n2):
                for c in range(n3):
                    # flat index of (m - m') mod n for every m, with m' = (a, b, c)
                    self._shift.append(np.roll(idx, shift=(a, b, c), axis=(0, 1, 2)).reshape(-1))

    def FT(self, f):
        return np.array(f, dtype=np.complex128, copy=True)

    def iFT(self, F):
        return np.array(F, dtype=np.complex128, copy=True)

    def mul(self, a, b):
        a, b = np.broadcast_arrays(a, b)
        shp = a.shape
        A = a.reshape(shp[:-3] + (self.N,))
        Bf = b.reshape(shp[:-3] + (self.N,))
        out = np.zeros_like(A)
        for mp in range(self.N):
            out += A[..., mp : mp + 1] * Bf[..., self._shift[mp]]
        return out.reshape(shp)

    def conj(self, a):
        return np.conj(self.spec_neg(a))

    def const(self, value):
        out = np.zeros(self.n, dtype=np.complex128)
        out[0, 0, 0] = value
        return out

    def orbital(self, c, k):
        return self.box(c, k)

    def orbital_grad(self, c, k):
        kg = self.S.kpG(k)
        npw = self.S.npw[k]
        g = 1j * c[..., None, :npw] * kg.T[None] if c.ndim == 2 else 1j * c[None, :npw] * kg.T
        return self.box(g, k)

    def project(self, f, k):
        i0, i1, i2 = self.S.box_index[k]
        out = np.zeros(f.shape[:-3] + (self.S.npw_max,), dtype=np.complex128)
        out[..., : self.S.npw[k]] = f[..., i0, i1, i2]
        return out
