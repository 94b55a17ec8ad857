"""Pins of the crystal-symmetry oracle (Sec. 2.3 end, Sec. 2.6.4 symmetry relations).

The unfolding of orbitals is checked against an independent construction --
the model operator diagonalised directly at every k-point -- and the
symmetry-reduced occupied-pair stage against the full one, which needs no
symmetry at all.  A non-symmetric input shows the reduction is not a no-op.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import operator as OP
from oracle import symmetry as SY
from paper_2302_07420_gb300 import synth


def _case(kmesh, fft, ecut):
    p = synth.si_params(kmesh=kmesh, fft=fft, ecut=ecut)
    S = make_setup(p)
    ops = synth.point_group(p["lattice"])
    kinfo, irred = SY.kmap(ops, S.kfrac, True)
    cp, cc, eig, gap = synth.model_orbitals(p["lattice"], S.kcart, S.miller, S.npw_max, 4)
    assert gap > 0.05
    return p, S, ops, kinfo, irred, cp, cc


def test_point_groups():
    p = synth.si_params()
    full = synth.point_group(p["lattice"], atoms_frac=((0.0, 0.0, 0.0),))
    dia = synth.point_group(p["lattice"])
    assert len(full) == 48 and len(dia) == 24            # O_h of the fcc lattice, T_d of the diamond basis
    for ops in (full, dia):
        np.testing.assert_array_equal(ops[0], np.eye(3, dtype=np.int64))
        keys = {tuple(S.ravel()) for S in ops}
        for A in ops:                                     # closure
            for B in ops:
                assert tuple((A @ B).ravel()) in keys
        L = p["lattice"]
        for S in ops:                                     # Cartesian forms are orthogonal
            Sc = L.T @ S @ np.linalg.inv(L.T)
            np.testing.assert_allclose(Sc @ Sc.T, np.eye(3), atol=1e-12)


def test_cartesian_forms_on_a_non_symmetric_basis():
    """x -> S x on fractional coordinates is r -> L^T S L^-T r in Cartesian ones (rows a_i of L): the
    Cartesian form of every operation that keeps the metric is orthogonal, also for a basis whose matrix
    is not symmetric (the fcc cell with a_3 replaced by a_1 + a_3), and a proper rotation for det S = 1."""
    L = np.array([[1, 0, 0], [0, 1, 0], [1, 0, 1]]) @ synth.si_params()["lattice"]
    assert np.abs(L - L.T).max() > 1.0
    Sset = type("Cell", (), {"lattice": L})()
    ops = synth.point_group(L, atoms_frac=((0.0, 0.0, 0.0),))
    assert len(ops) >= 8
    for S in ops:
        R = SY.cart(Sset, S)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - np.linalg.det(S)) < 1e-12
        np.testing.assert_allclose(R @ L.T, L.T @ S, atol=1e-12)      # maps the rotated lattice vectors


def test_kmap_takes_the_first_operation_in_order():
    """Each irreducible point is its own image under the identity (operation 0, no time reversal, K = 0),
    and every other point records the first operation, in the stated order (all operations without time
    reversal, then all with it), that reaches it from its irreducible point."""
    p = synth.si_params(kmesh=(4, 4, 4))
    S = make_setup(p)
    ops = synth.point_group(p["lattice"])
    kinfo, irred = SY.kmap(ops, S.kfrac, True)
    for k0 in irred:
        assert kinfo[k0][0] == k0 and kinfo[k0][1] == 0 and kinfo[k0][2] == 1 and not np.any(kinfo[k0][3])
    order = [(tr, s) for tr in (1, -1) for s in range(len(ops))]
    for k, (k0, s, tr, K) in enumerate(kinfo):
        for tr2, s2 in order[: order.index((tr, s))]:
            d = tr2 * (ops[s2].T @ S.kfrac[k0]) - S.kfrac[k]
            assert not np.all(np.abs(d - np.round(d)) < 1e-9), (k, tr2, s2)


@pytest.mark.parametrize("kmesh,nirr", [((4, 4, 4), 8), ((2, 2, 2), 3), ((3, 3, 3), 4)])
def test_irreducible_k_points(kmesh, nirr):
    """T_d with time reversal acts on k like O_h (time reversal supplies the inversion): the same
    irreducible count as O_h with or without time reversal (8 for the Gamma-centred 4x4x4 fcc mesh,
    Gamma, L, X for 2x2x2); every star has |G| / |stabiliser| points."""
    p = synth.si_params(kmesh=kmesh)
    S = make_setup(p)
    dia = synth.point_group(p["lattice"])
    oh = synth.point_group(p["lattice"], atoms_frac=((0.0, 0.0, 0.0),))
    counts = [len(SY.kmap(ops, S.kfrac, tr)[1]) for ops, tr in ((dia, True), (oh, False), (oh, True))]
    assert counts == [nirr] * 3
    kinfo, irred = SY.kmap(dia, S.kfrac, True)
    for k, (k0, s, tr, K) in enumerate(kinfo):
        np.testing.assert_allclose(tr * (dia[s].T @ S.kfrac[k0]) - K, S.kfrac[k], atol=1e-12)
        assert k0 in irred
    for k0 in irred:
        stab = 0
        for tr in (1, -1):
            for Sop in dia:
                d = tr * (Sop.T @ S.kfrac[k0]) - S.kfrac[k0]
                stab += int(np.all(np.abs(d - np.round(d)) < 1e-9))
        assert sum(1 for x in kinfo if x[0] == k0) == 2 * len(dia) // stab


@pytest.mark.parametrize("kmesh,fft,ecut", [((2, 2, 2), 16, 3.0), ((3, 3, 3), 15, 2.5)])
def test_unfolded_orbitals_span_the_model_eigenspaces(kmesh, fft, ecut):
    """The rotated (and, where used, time-reversed and K-shifted) irreducible orbitals give the same
    right/left projectors as the model operator diagonalised at each k directly."""
    p, S, ops, kinfo, irred, cp, cc = _case(kmesh, fft, ecut)
    assert any(x[2] < 0 for x in kinfo) or kmesh == (2, 2, 2)
    up = SY.unfold_orbitals(S, cp, ops, kinfo)
    uc = SY.unfold_orbitals(S, cc, ops, kinfo)
    for k in range(S.Nk):
        np.testing.assert_allclose(up[k].T @ np.conj(uc[k]), cp[k].T @ np.conj(cc[k]), atol=1e-13)
        np.testing.assert_allclose(np.conj(uc[k]) @ up[k].T, np.eye(4), atol=1e-13)
    if kmesh == (2, 2, 2):
        assert any(np.any(x[3]) for x in kinfo)           # a K shift is exercised


@pytest.mark.parametrize("kmesh,left", [((2, 2, 2), False), ((3, 3, 3), True)])
def test_reduced_occupied_pair_stage_equals_the_full_one(kmesh, left):
    p, S, ops, kinfo, irred, cp, cc = _case(kmesh, 12, 1.5)
    up = SY.unfold_orbitals(S, cp, ops, kinfo)
    uc = SY.unfold_orbitals(S, cc, ops, kinfo)
    occ = synth.occupations(S.Nk, 4, 4)
    full = OP.TCOperator(S, up, uc, occ, left=left)
    red = OP.TCOperator(S, up, uc, occ, left=left, sym=(ops, kinfo, irred))
    full.prepare()
    red.prepare()
    for name in ("h6", "h5"):
        a, b = getattr(full, name), getattr(red, name)
        assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    for k in range(S.Nk):
        for name in ("h3a4", "h3b"):
            a, b = getattr(full, name)[k], getattr(red, name)[k]
            assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    rf, rr = full.apply(), red.apply()
    sc = max(np.abs(v).max() for v in rf.values())
    for t in OP.TERMS:
        assert np.abs(rf[t] - rr[t]).max() < 1e-13 * sc, t


def test_reduction_is_not_a_no_op_on_non_symmetric_orbitals():
    p = synth.si_params(kmesh=(2, 2, 2), fft=12, ecut=1.5)
    S = make_setup(p)
    ops = synth.point_group(p["lattice"])
    kinfo, irred = SY.kmap(ops, S.kfrac, True)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 800, [S.kpG(k) for k in range(S.Nk)], S.npw_max, 4,
                                         perturb=0.1)
    occ = synth.occupations(S.Nk, 4, 4)
    full = OP.total(OP.apply_operator(S, c_phi, c_chi, occ))
    red = OP.total(OP.apply_operator(S, c_phi, c_chi, occ, sym=(ops, kinfo, irred)))
    assert np.abs(full - red).max() > 1e-3 * np.abs(full).max()
