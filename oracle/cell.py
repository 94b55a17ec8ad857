"""Cell, k mesh, plane-wave spheres and the divergence-correction constant (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions (arXiv:2302.07420):

* lattice rows a_i (bohr); reciprocal rows b_i with a_i . b_j = 2 pi delta_ij.
* Gamma-centred Monkhorst-Pack mesh (the paper's QE inputs use "n n n 0 0 0",
  Sec. 4); fractional coordinates are taken in (-1/2, 1/2]; k index
  ``(i1*N2 + i2)*N3 + i3``.
* plane-wave sphere at k: all Miller vectors m with |k + m.B|^2 / 2 <= ecut
  (Hartree), ordered lexicographically by (m1, m2, m3).
* FFT box n1 x n2 x n3, real-space point r = sum_i (i_i / n_i) a_i.  FFT index
  m_i in [0, n_i) stands for the Miller integer ``rep(m_i)`` of numpy's fftfreq
  convention (m_i if m_i <= (n_i-1)//2 else m_i - n_i).
* periodic Fourier transform with the 1/Omega convention of Sec. 2.2, which on
  the grid is FT[f](G) = (1/N) sum_r f(r) e^{-iG.r}, FT^{-1}[F](r) = sum_G F(G) e^{iG.r}.

Divergence correction (Sec. 2.5): with the auxiliary function
A_aux(q) = exp(-alpha q^2)/q^2 (Eq. aux) and k on the SCF mesh, the bracket of
Eq. correction2 is

    Gamma0 = Omega / (4 sqrt(pi^3 alpha)) - (1/N_k) (-alpha + sum'_{q,G} A_aux(k - q + G)),

which does not depend on k when k is a mesh point.  The paper gives no value
for alpha; the reading used here is sqrt(alpha) = L_min / 12 with L_min the
shortest lattice vector of the Born-von Karman supercell, and the primed sum
runs over every reciprocal vector of that supercell until exp(-alpha p^2) < 1e-20.

Parity pins: sphere counts on the cutoff (inclusive; lattice-point counts of
the simple-cubic cell), sizes and ordering compared bit-exactly with the CUDA
library's layout; Gamma0 is pinned by an independent Ewald sum (4 pi Gamma0 /
Omega = -v_Madelung of the supercell) and by the simple-cubic Madelung constant.
"""
import numpy as np

ALPHA_TAIL = 1e-20


def reciprocal(lattice):
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    lattice = np.asarray(lattice, dtype=np.float64)
    return 2.0 * np.pi * np.linalg.inv(lattice).T


def kmesh_frac(kmesh):
    """Gamma-centred mesh, fractional coordinates in (-1/2, 1/2], shape (Nk, 3)."""
    axes = []
    for n in kmesh:
        f = np.arange(n, dtype=np.float64) / n
        f = np.where(f > 0.5, f - 1.0, f)
        axes.append(f)
    g = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


def sphere_miller(kcart, B, ecut):
    """Miller vectors m (npw, 3) of the sphere |k + m.B|^2/2 <= ecut, lexicographic."""
    gmax = np.sqrt(2.0 * ecut) + np.linalg.norm(kcart)
    lat = np.linalg.inv(B).T * 2.0 * np.pi       # rows a_i
    bound = [int(np.ceil(gmax * np.linalg.norm(lat[i]) / (2.0 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-b, b + 1) for b in bound]
    m = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    kg = kcart[None, :] + m @ B
    keep = 0.5 * np.einsum("ij,ij->i", kg, kg) <= ecut
    return m[keep]                               # meshgrid 'ij' order is lexicographic


def fft_rep(n):
    """Miller integer represented by each FFT index 0..n-1 (numpy fftfreq convention)."""
    i = np.arange(n)
    return np.where(i <= (n - 1) // 2, i, i - n)


def shortest_supercell_vector(lattice, kmesh):
    S = np.asarray(lattice, dtype=np.float64) * np.asarray(kmesh, dtype=np.float64)[:, None]
    best = np.inf
    r = range(-2, 3)
    for i in r:
        for j in r:
            for k in r:
                if i == j == k == 0:
                    continue
                v = i * S[0] + j * S[1] + k * S[2]
                best = min(best, float(np.linalg.norm(v)))
    return best


def default_alpha(lattice, kmesh):
    return (shortest_supercell_vector(lattice, kmesh) / 12.0) ** 2


def aux_sum(lattice, kmesh, alpha):
    """sum' of exp(-alpha p^2)/p^2 over the supercell reciprocal lattice (p != 0)."""
    B = reciprocal(lattice)
    kmesh = np.asarray(kmesh)
    Bs = B / kmesh[:, None]                      # supercell reciprocal rows b_i / N_i
    pmax = np.sqrt(-np.log(ALPHA_TAIL) / alpha)
    S = np.asarray(lattice, dtype=np.float64) * kmesh[:, None]
    bound = [int(np.ceil(pmax * np.linalg.norm(S[i]) / (2.0 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-b, b + 1) for b in bound]
    l = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    p = l @ Bs
    p2 = np.einsum("ij,ij->i", p, p)
    p2 = p2[p2 > 0.0]
    w = np.exp(-alpha * p2) / p2
    return float(np.sum(np.sort(w)))             # ascending order for a stable sum


def gamma0(lattice, kmesh, alpha):
    """Bracket of Eq. correction2 for k on the SCF mesh."""
    Omega = abs(np.linalg.det(np.asarray(lattice, dtype=np.float64)))
    Nk = int(np.prod(kmesh))
    return Omega / (4.0 * np.sqrt(np.pi ** 3 * alpha)) - (-alpha + aux_sum(lattice, kmesh, alpha)) / Nk


class Setup:
    """Everything ``tc_init`` fixes: geometry, basis, box maps and constants."""

    def __init__(self, lattice, kmesh, ecut, fft, nbands, nocc, A, C,
                 alpha=0.0, div_correction=1, ushort_factor=1.0):
        self.lattice = np.asarray(lattice, dtype=np.float64)
        self.B = reciprocal(self.lattice)
        self.Omega = abs(float(np.linalg.det(self.lattice)))
        self.kmesh = tuple(int(x) for x in kmesh)
        self.Nk = int(np.prod(self.kmesh))
        self.kfrac = kmesh_frac(self.kmesh)
        self.kcart = self.kfrac @ self.B
        self.ecut = float(ecut)
        self.n = tuple(int(x) for x in fft)
        self.N = int(np.prod(self.n))
        self.nbands = int(nbands)
        self.nocc = int(nocc)
        self.A = np.asarray(A, dtype=np.float64)    # [pp, ap]
        self.C = np.asarray(C, dtype=np.float64)    # [pp, ap]
        self.alpha = float(alpha) if alpha > 0 else default_alpha(self.lattice, self.kmesh)
        self.div_correction = int(div_correction)
        self.ushort_factor = float(ushort_factor)
        if not (0 < self.nocc <= self.nbands):
            raise ValueError("need 0 < nocc <= nbands")

        self.miller = [sphere_miller(self.kcart[k], self.B, self.ecut) for k in range(self.Nk)]
        self.npw = np.array([len(m) for m in self.miller], dtype=np.int64)
        self.npw_max = int(self.npw.max())
        for m in self.miller:
            for i in range(3):
                if np.abs(m[:, i]).max() > (self.n[i] - 1) // 2:
                    raise ValueError("plane-wave sphere does not fit the FFT box")
        # box index of each sphere element, per k
        self.box_index = [tuple((m[:, i] % self.n[i]) for i in range(3)) for m in self.miller]
        rep = [fft_rep(n) for n in self.n]
        R = np.stack(np.meshgrid(*rep, indexing="ij"), axis=-1).astype(np.float64)
        self.Gbox = R @ self.B                        # (n1, n2, n3, 3) Cartesian G of each index
        self.Gamma0 = gamma0(self.lattice, self.kmesh, self.alpha)

    def kpG(self, k):
        """Cartesian k+G over the sphere of k-point k, shape (npw, 3)."""
        return self.kcart[k][None, :] + self.miller[k] @ self.B
