"""Seeded synthetic inputs (cells, parameters, orbitals) for the TC operator.

This module holds input recipes only -- no step of the operator itself.  The
caller supplies the plane-wave basis (Miller vectors and k+G per k-point); the
module draws coefficients on it.  Seeds are 230207420 + workload index.

Workloads (all in Hartree atomic units):

* ``heg_14``   -- homogeneous electron gas, simple-cubic cell, N = 14 electrons
  (7 doubly occupied plane waves n in {0, +-e_x, +-e_y, +-e_z}), r_s = 4,
  Gamma only, FFT box 16^3, sphere |n|^2 <= 16; chi = phi.
* ``si_k444``  -- silicon-like FCC cell, a = 10.26 bohr, 8 electrons (4 occupied
  bands per k), 4x4x4 Gamma-centred mesh, ecut = 7.5 Ha (15 Ry), box 24^3.
  Coefficients (N(0,1) + i N(0,1))/sqrt(2) exp(-|k+G|^2/4), orthonormalised per
  k by modified Gram-Schmidt (band order); chi = X' (Phi^H X')^{-1} with X' = Phi + 1e-2 R (R drawn the same way,
  column-normalised), so chi^H phi = I and <phi_i|phi_i> = 1.
* ``heg_114``  -- HEG, N = 114 electrons (57 plane waves, |n|^2 <= 5), r_s = 2,
  Gamma only, box 48^3, sphere |n|^2 <= 144.
* ``tiny_*``   -- small random cells for brute-force checks.
* ``heg_batch`` -- many independent HEG cells of uneven size (box 16^3-32^3,
  1-8 k-points, 7-33 occupied plane waves per k), see ``heg_batch``.

Jastrow parameters follow Eqs. A_normalize and cusp: A = sqrt(Omega/(4 pi N)),
C_pp = sqrt(2 A), C_ap = sqrt(A).
"""
import numpy as np

SEED0 = 230207420


def jastrow_params(Omega, nelec, A=None):
    if A is None:
        A = np.sqrt(Omega / (4.0 * np.pi * nelec))
    return [A, A], [np.sqrt(2.0 * A), np.sqrt(A)]


def heg_params(nelec, rs, fft, radius2):
    L = (nelec * 4.0 * np.pi / 3.0) ** (1.0 / 3.0) * rs
    lattice = np.eye(3) * L
    Omega = L ** 3
    b = 2.0 * np.pi / L
    ecut = 0.5 * radius2 * b * b * (1.0 + 1e-9)
    A, C = jastrow_params(Omega, nelec)
    nocc = nelec // 2
    return dict(lattice=lattice, kmesh=(1, 1, 1), ecut=ecut, fft=(fft,) * 3, nbands=nocc,
                nocc=nocc, A=A, C=C, nelec=nelec)


def si_params(kmesh=(4, 4, 4), fft=24, ecut=7.5, nbands=4, nocc=4):
    a = 10.26
    lattice = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    Omega = abs(np.linalg.det(lattice))
    A, C = jastrow_params(Omega, 8)
    return dict(lattice=lattice, kmesh=tuple(kmesh), ecut=ecut, fft=(fft,) * 3, nbands=nbands,
                nocc=nocc, A=A, C=C, nelec=8)


def tiny_params(seed, kmesh=(1, 1, 2), fft=(8, 9, 10), ecut=1.2, nbands=3, nocc=2, scale=6.0):
    """A slightly distorted triclinic cell, for brute-force and invariance checks."""
    rng = np.random.default_rng(SEED0 + 100 + seed)
    lattice = scale * (np.eye(3) + 0.15 * rng.standard_normal((3, 3)))
    Omega = abs(np.linalg.det(lattice))
    A, C = jastrow_params(Omega, 2 * nocc)
    return dict(lattice=lattice, kmesh=tuple(kmesh), ecut=ecut, fft=tuple(fft), nbands=nbands,
                nocc=nocc, A=A, C=C, nelec=2 * nocc)


WORKLOADS = {
    "heg_14": lambda: heg_params(14, 4.0, 16, 16),
    "si_k444": lambda: si_params(),
    "heg_114": lambda: heg_params(114, 2.0, 48, 144),
}


def _gauss_coeffs(rng, kpg, npw_max, nbands):
    npw = kpg.shape[0]
    damp = np.exp(-np.einsum("ij,ij->i", kpg, kpg) / 4.0)
    c = (rng.standard_normal((npw, nbands)) + 1j * rng.standard_normal((npw, nbands))) / np.sqrt(2.0)
    return c * damp[:, None]


def _gram_schmidt(P):
    """Modified Gram-Schmidt on the columns (platform-independent signs)."""
    P = P.copy()
    for b in range(P.shape[1]):
        for a in range(b):
            P[:, b] -= np.vdot(P[:, a], P[:, b]) * P[:, a]
        P[:, b] /= np.linalg.norm(P[:, b])
    return P


def random_orbitals(seed, kpg_list, npw_max, nbands, perturb=1e-2):
    """(c_phi, c_chi) of shape (Nk, nbands, npw_max), biorthonormal per k.

    ``kpg_list[k]`` is the (npw_k, 3) array of Cartesian k+G of the sphere at k.
    """
    rng = np.random.default_rng(seed)
    Nk = len(kpg_list)
    c_phi = np.zeros((Nk, nbands, npw_max), dtype=np.complex128)
    c_chi = np.zeros_like(c_phi)
    for k, kpg in enumerate(kpg_list):
        npw = kpg.shape[0]
        P = _gram_schmidt(_gauss_coeffs(rng, kpg, npw_max, nbands))
        R = _gauss_coeffs(rng, kpg, npw_max, nbands)
        R = R / np.linalg.norm(R, axis=0, keepdims=True)
        Xp = P + perturb * R
        X = Xp @ np.linalg.inv(P.conj().T @ Xp)
        c_phi[k, :, :npw] = P.T
        c_chi[k, :, :npw] = X.T
    return c_phi, c_chi


def heg_orbitals(miller0, npw_max, radius2_occ):
    """Unit plane waves on all Miller vectors with |n|^2 <= radius2_occ (Gamma only).

    Orbitals are ordered by (|n|^2, n1, n2, n3); returns c (1, nocc, npw_max).
    """
    m = np.asarray(miller0)
    r2 = np.einsum("ij,ij->i", m, m)
    sel = np.nonzero(r2 <= radius2_occ)[0]
    order = sorted(sel, key=lambda i: (r2[i], m[i, 0], m[i, 1], m[i, 2]))
    c = np.zeros((1, len(order), npw_max), dtype=np.complex128)
    for b, i in enumerate(order):
        c[0, b, i] = 1.0
    return c


def heg_kpoint_orbitals(kpg_list, miller_list, npw_max, nocc):
    """Unit plane waves e^{i(k+G).r}: at every k the nocc lowest |k+G|^2 of the sphere.

    Ties are broken by (|k+G|^2, m1, m2, m3); returns c (Nk, nocc, npw_max).
    """
    Nk = len(kpg_list)
    c = np.zeros((Nk, nocc, npw_max), dtype=np.complex128)
    for k in range(Nk):
        kpg, m = np.asarray(kpg_list[k]), np.asarray(miller_list[k])
        q2 = np.einsum("ij,ij->i", kpg, kpg)
        order = sorted(range(len(q2)), key=lambda i: (round(q2[i], 12), m[i, 0], m[i, 1], m[i, 2]))
        if len(order) < nocc:
            raise ValueError("sphere holds fewer plane waves than occupied bands")
        for b, i in enumerate(order[:nocc]):
            c[k, b, i] = 1.0
    return c


HEG_BATCH_N = (14, 38, 54, 66)
HEG_BATCH_BOX = (16, 18, 20, 24, 25, 27, 30, 32)
HEG_BATCH_KMESH = ((1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2))


def heg_batch(ncell=256, index=4):
    """Independent HEG cells: N uniform in {14, 38, 54, 66}, r_s uniform in [1, 5],
    box uniform in {16, 18, 20, 24, 25, 27, 30, 32}, k mesh uniform in
    {1x1x1, 1x1x2, 1x2x2, 2x2x2}; nbands = nocc = N/2, plane-wave sphere
    |m|_2 <= floor((n - 1)/4) in index units (r = floor((n-1)/4)), A and C from
    Eqs. A_normalize and cusp.  Seed 230207420 + index."""
    rng = np.random.default_rng(SEED0 + index)
    cells = []
    for _ in range(ncell):
        nelec = int(rng.choice(HEG_BATCH_N))
        rs = float(rng.uniform(1.0, 5.0))
        n = int(rng.choice(HEG_BATCH_BOX))
        kmesh = tuple(HEG_BATCH_KMESH[int(rng.integers(len(HEG_BATCH_KMESH)))])
        r = (n - 1) // 4
        p = heg_params(nelec, rs, n, r * r)
        p["kmesh"] = kmesh
        p["ecut"] = 0.5 * (r * 2.0 * np.pi / p["lattice"][0, 0]) ** 2 * (1.0 + 1e-9)
        cells.append(p)
    return cells


def occupations(Nk, nbands, nocc, fill=1.0):
    occ = np.zeros((Nk, nbands))
    occ[:, :nocc] = fill
    return occ


# ---------------------------------------------------------------------------
# Crystal-symmetric inputs.  Orbitals that obey the point group of a crystal
# come from diagonalising a model one-body operator that has that symmetry:
#   h(k)_{GG'} = |k+G|^2/2 delta_GG' + V(G - G') - lam W(G - G') (G - G').(k + G'),
#   V(Q) = v0 (|Q|^2 - qc2) exp(-|Q|^2/sv^2) s(Q),  W(Q) = w0 exp(-|Q|^2/sw^2) s(Q),
#   s(Q) = (1/n_at) sum_atoms exp(-i Q.tau_a),
# i.e. T + V(r) + lam grad W(r) . grad with V, W sums of spherical atomic
# functions: real in real space (time-reversal symmetric) and non-Hermitian
# for lam != 0 (a TC-like first-order term).  Right / left eigenvectors of the
# nbands eigenvalues of lowest real part, per k-point, give phi (Gram-Schmidt)
# and chi (biorthonormal to phi); a gap after band nbands at every k-point
# makes the occupied spaces symmetric.

SI_ATOMS = ((0.0, 0.0, 0.0), (0.25, 0.25, 0.25))   # diamond structure, fractional coordinates


def point_group(lattice, atoms_frac=SI_ATOMS):
    """Integer matrices S (x -> S x on fractional real-space coordinates) that keep the
    lattice metric and map the atom set onto itself (modulo lattice vectors); identity first."""
    import itertools
    L = np.asarray(lattice, dtype=np.float64)
    M = L @ L.T
    cand = np.array(list(itertools.product((-1, 0, 1), repeat=9)), dtype=np.int64).reshape(-1, 3, 3)
    lhs = np.einsum("nji,jk,nkl->nil", cand, M, cand)
    keep = np.all(np.abs(lhs - M[None]) <= 1e-9 * np.abs(M).max(), axis=(1, 2))
    cand = cand[keep]
    X = np.asarray(atoms_frac, dtype=np.float64)
    ops = []
    for S in cand:
        Y = X @ S.T
        ok = True
        for y in Y:
            d = X - y[None]
            if not np.any(np.all(np.abs(d - np.round(d)) < 1e-9, axis=1)):
                ok = False
                break
        if ok:
            ops.append(S)
    ops.sort(key=lambda S: (0 if np.array_equal(S, np.eye(3, dtype=np.int64)) else 1, tuple(S.ravel())))
    return np.array(ops, dtype=np.int64)


MODEL = dict(v0=0.16, qc2=2.0, sv=1.5, w0=0.05, sw=1.5, lam=1.0)


def model_orbitals(lattice, kcart, miller_list, npw_max, nbands, atoms_frac=SI_ATOMS, model=None):
    """(c_phi, c_chi, eig (Nk, nbands+1) complex, gap): symmetric model orbitals on the given spheres.

    kcart: (Nk, 3) Cartesian k; miller_list[k]: (npw_k, 3) Miller indices of the sphere.
    gap = min over k of Re eig[nbands] - Re eig[nbands-1] (must be > 0 for symmetric occupied spaces).
    """
    prm = dict(MODEL, **(model or {}))
    L = np.asarray(lattice, dtype=np.float64)
    B = 2.0 * np.pi * np.linalg.inv(L).T
    tau = np.asarray(atoms_frac, dtype=np.float64) @ L
    Nk = len(miller_list)
    c_phi = np.zeros((Nk, nbands, npw_max), dtype=np.complex128)
    c_chi = np.zeros_like(c_phi)
    eig = np.zeros((Nk, nbands + 1), dtype=np.complex128)
    gap = np.inf
    for k in range(Nk):
        G = np.asarray(miller_list[k], dtype=np.float64) @ B
        kG = kcart[k][None] + G
        Q = G[:, None, :] - G[None, :, :]
        q2 = np.einsum("ijd,ijd->ij", Q, Q)
        sf = np.mean(np.exp(-1j * np.einsum("ijd,ad->ija", Q, tau)), axis=2)
        V = prm["v0"] * (q2 - prm["qc2"]) * np.exp(-q2 / prm["sv"] ** 2) * sf
        W = prm["w0"] * np.exp(-q2 / prm["sw"] ** 2) * sf
        H = V - prm["lam"] * W * np.einsum("ijd,jd->ij", Q, kG)
        H[np.diag_indices_from(H)] += 0.5 * np.einsum("id,id->i", kG, kG)
        lam_, Y = np.linalg.eig(H)
        order = np.argsort(lam_.real, kind="stable")
        lam_, Y = lam_[order], Y[:, order]
        Z = np.linalg.inv(Y).conj().T
        eig[k] = lam_[: nbands + 1]
        gap = min(gap, lam_[nbands].real - lam_[nbands - 1].real)
        P = _gram_schmidt(Y[:, :nbands])
        Xp = Z[:, :nbands]
        X = Xp @ np.linalg.inv(P.conj().T @ Xp)
        n = G.shape[0]
        c_phi[k, :, :n] = P.T
        c_chi[k, :, :n] = X.T
    return c_phi, c_chi, eig, gap
