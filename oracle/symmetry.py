"""Crystal symmetry for the k mesh, the orbitals and the occupied-pair fields (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.3 (end): a symmorphic operation r -> S r (t = 0) maps the orbital of
k0 onto one of k = S^dagger k0, with coefficients phi~_k(S^dagger G0) =
phi~_k0(G0); with time reversal k = -S^dagger k0 and the coefficients are
conjugated.  Sec. 2.6.4 uses the same operations to obtain the occupied-pair
fields of every q2 from those of the irreducible q2;0 (the text after Alg. 4
and Eqs. symope_3a2_1 / symope_3a2_2):
  h5~(S^dagger G; q2) = h5~(G; q2;0),      h3~(S^dagger G; q2) = S^dagger h3~(G; q2;0),
and with time reversal
  h5~(-S^dagger G; q2) = conj h5~(G; q2;0), h3~(-S^dagger G; q2) = +S^dagger conj h3~(G; q2;0).
The time-reversed vector relation is printed with -S^dagger; for h3 as Algs. 6
and 8 define it -- with the factor i of the grad-u kernel i p u~(p) inside --
the conjugation contributes a second sign (conj(i) = -i) that cancels the
sign of the reversed argument, so the relation holds with +S^dagger (the
full computation pins this).

Conventions.  S is an integer matrix acting on fractional real-space
coordinates (x -> S x); its Cartesian form is S_c = L^T S L^-T (L: rows a_i),
so S^dagger = S_c^T.  In Miller indices G = B^T m, S^dagger G = B^T (S^T m),
and a k-point with reciprocal fractional coordinates kappa maps to S^T kappa.
Mesh points carry coordinates in (-1/2, 1/2], so the image of k0 is a mesh
point k up to a reciprocal lattice vector K: k = +-S^T k0 - K.  The cell-periodic
part then picks up e^{i K.r}; in Miller indices (reading of the printed
relation, which assumes K = 0):
  no time reversal:  phi~_k(S^T m0 + K) = phi~_k0(m0)
  time reversal:     phi~_k(-S^T m0 + K) = conj phi~_k0(m0).
A field whose crystal momentum is +k2 (h3 of 3a4: P(q1,q2) phi_q1) shifts by
+K, one with momentum -k2 (h3 of 3b2/3b5: P(q2,q1) chi_q1^*) by -K, and the
h6 contribution of q2 (momentum 0) does not shift.

The map takes the mesh points in order; a point not reached from an earlier
irreducible point is irreducible itself, and every operation (then, with time
reversal, every operation times -1) is tried on it in the given order; the
first one to reach a point assigns it.

Parity pins (tests/test_oracle_symmetry.py): the unfolded model orbitals
span the occupied eigenspaces of the model operator built directly at each
k; the symmetry-reduced occupied-pair stage reproduces the full one (h6,
both h3 kinds, every operator term) on unfolded orbitals and not on
non-symmetric ones; group closure and the size of the irreducible set.
"""
import numpy as np


def kmap(ops, kfrac, time_reversal=True):
    """List of (k0, op, tr, K) per mesh point (tr = +1 or -1) and the irreducible indices."""
    kfrac = np.asarray(kfrac, dtype=np.float64)
    Nk = kfrac.shape[0]
    out = [None] * Nk
    irred = []
    signs = (1, -1) if time_reversal else (1,)
    for k0 in range(Nk):
        if out[k0] is not None:
            continue
        irred.append(k0)
        for tr in signs:
            for s, S in enumerate(ops):
                kap = tr * (np.asarray(S).T @ kfrac[k0])
                d = kap[None, :] - kfrac
                hit = np.nonzero(np.all(np.abs(d - np.round(d)) < 1e-9, axis=1))[0]
                if len(hit) != 1:
                    raise ValueError("operation does not map the k mesh onto itself")
                j = int(hit[0])
                if out[j] is None:
                    out[j] = (k0, s, tr, np.round(d[j]).astype(np.int64))
    return out, irred


def miller_image(S, tr, K, m0):
    """Miller indices of the image of m0 (rows): tr S^T m0 + K."""
    return tr * (np.asarray(m0) @ np.asarray(S)) + np.asarray(K)[None]


def unfold_orbitals(Sset, c, ops, kinfo):
    """Coefficients at every k from those of its irreducible point (Sec. 2.3)."""
    c = np.asarray(c, dtype=np.complex128)
    out = np.array(c)
    for k, (k0, s, tr, K) in enumerate(kinfo):
        if k == k0:
            continue
        img = miller_image(ops[s], tr, K, Sset.miller[k0])
        pos = {tuple(m): i for i, m in enumerate(Sset.miller[k])}
        if len(img) != Sset.npw[k]:
            raise ValueError("sphere sizes differ between symmetry-related k-points")
        out[k] = 0.0
        for i0, m in enumerate(img):
            i = pos[tuple(m)]
            v = c[k0, :, i0]
            out[k, :, i] = v if tr > 0 else np.conj(v)
    return out


def cart(Sset, S):
    """Cartesian form L^T S L^-T of a fractional operation."""
    L = Sset.lattice
    return L.T @ np.asarray(S, dtype=np.float64) @ np.linalg.inv(L.T)


def rotate_field(Sset, F_r, S, tr, K, vector):
    """Real-space field of q2 from that of q2;0 via its Fourier coefficients.

    F_r: (..., [3,] n1, n2, n3) real-space values; vector: the axis before the grid is a
    Cartesian component.  Coefficient at the image index tr S^T m0 + K (mod n) equals
    R F~(m0) (conjugated when tr = -1) with R = S_c^T for vectors, 1 for scalars.
    """
    n = np.array(Sset.n)
    N = int(np.prod(n))
    F = np.fft.fftn(F_r, axes=(-3, -2, -1)) / N
    grid = np.stack(np.meshgrid(*[np.arange(x) for x in n], indexing="ij"), axis=-1).reshape(-1, 3)
    img = np.mod(miller_image(S, tr, K, grid), n[None])
    G = np.zeros_like(F)
    src = F.reshape(F.shape[:-3] + (-1,))
    if tr < 0:
        src = np.conj(src)
    if vector:
        R = cart(Sset, S).T
        src = np.einsum("de,...ei->...di", R, src)
    dst = G.reshape(G.shape[:-3] + (-1,))
    flat = (img[:, 0] * n[1] + img[:, 1]) * n[2] + img[:, 2]
    dst[..., flat] = src
    return np.fft.ifftn(dst.reshape(G.shape), axes=(-3, -2, -1)) * N
