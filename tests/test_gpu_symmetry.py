"""Symmetry-reduced occupied-pair stage on the GPU against the oracle (Sec. 2.3 end, Sec. 2.6.4).

Inputs: orbitals of a model operator with the diamond structure's point group
(T_d, 24 operations) and time reversal, taken at the irreducible k-points and
unfolded to the rest of the mesh.  The reduced GPU operator must equal the
oracle's full operator (no symmetry used there) on those orbitals.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import operator as OP
from oracle import symmetry as SY
from paper_2302_07420_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(p, **kw):
    from paper_2302_07420_gb300.operator import Context
    args = dict(lattice=p["lattice"], kmesh=p["kmesh"], ecut=p["ecut"], fft=p["fft"], nbands=p["nbands"],
                nocc=p["nocc"], A=p["A"], C=p["C"])
    args.update(kw)
    return Context(**args)


def _inputs(kmesh, fft, ecut):
    p = synth.si_params(kmesh=kmesh, fft=fft, ecut=ecut)
    S = make_setup(p)
    ops = synth.point_group(p["lattice"])
    kinfo, irred = SY.kmap(ops, S.kfrac, True)
    cp, cc, eig, gap = synth.model_orbitals(p["lattice"], S.kcart, S.miller, S.npw_max, 4)
    assert gap > 0.05
    up = SY.unfold_orbitals(S, cp, ops, kinfo)
    uc = SY.unfold_orbitals(S, cc, ops, kinfo)
    return p, S, ops, kinfo, irred, cp, cc, up, uc


@pytest.mark.parametrize("kmesh", [(4, 4, 4), (3, 3, 3), (2, 2, 2)])
def test_k_map_matches_the_oracle(kmesh):
    p = synth.si_params(kmesh=kmesh)
    S = make_setup(p)
    ops = synth.point_group(p["lattice"])
    kinfo, irred = SY.kmap(ops, S.kfrac, True)
    ctx = _ctx(p)
    try:
        ctx.set_symmetry(ops)
        nirr, km = ctx.symmetry_info()
    finally:
        ctx.close()
    assert nirr == len(irred)
    ref = np.array([[k0, s, tr, *K] for (k0, s, tr, K) in kinfo])
    np.testing.assert_array_equal(km, ref)


def test_symmetrize_orbitals_is_the_oracle_unfolding():
    p, S, ops, kinfo, irred, cp, cc, up, uc = _inputs((3, 3, 3), 15, 2.5)
    ctx = _ctx(p)
    try:
        ctx.set_symmetry(ops)
        a, b = torch.from_numpy(cp.copy()).cuda(), torch.from_numpy(cc.copy()).cuda()
        ctx.symmetrize_orbitals(a, b)
        torch.cuda.synchronize()
        h1, h2 = cp.copy(), cc.copy()
        ctx.symmetrize_orbitals(h1, h2)                   # host arrays
    finally:
        ctx.close()
    np.testing.assert_array_equal(a.cpu().numpy(), up)
    np.testing.assert_array_equal(b.cpu().numpy(), uc)
    np.testing.assert_array_equal(h1, up)
    np.testing.assert_array_equal(h2, uc)


@pytest.mark.parametrize("kmesh,prec,tol", [((2, 2, 2), "fp64", 1e-11), ((3, 3, 3), "fp64", 1e-11),
                                            ((3, 3, 3), "fp32", 1e-5)])
def test_reduced_apply_matches_the_full_oracle(kmesh, prec, tol):
    p, S, ops, kinfo, irred, cp, cc, up, uc = _inputs(kmesh, 12, 1.5)
    occ = synth.occupations(S.Nk, 4, 4)
    ref_r, ref_l = OP.tc_apply(S, up, uc, occ)
    ctx = _ctx(p, precision=prec)
    try:
        ctx.set_symmetry(ops)
        r, l = ctx.apply(torch.from_numpy(up).cuda(), torch.from_numpy(uc).cuda(), occ)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    sc = max(np.abs(ref_r).max(), np.abs(ref_l).max())
    assert np.abs(r.cpu().numpy() - ref_r).max() / sc < tol
    assert np.abs(l.cpu().numpy() - ref_l).max() / sc < tol


def test_reduced_energy_matches_the_unreduced_one():
    p, S, ops, kinfo, irred, cp, cc, up, uc = _inputs((2, 2, 2), 16, 3.0)
    occ = synth.occupations(S.Nk, 4, 4)
    ctx = _ctx(p)
    try:
        a, b = torch.from_numpy(up).cuda(), torch.from_numpy(uc).cuda()
        e_full = ctx.energy(a, b, occ)
        ctx.set_symmetry(ops)
        e_sym = ctx.energy(a, b, occ)
        ctx.set_symmetry([])                              # off again: the full stage
        e_off = ctx.energy(a, b, occ)
    finally:
        ctx.close()
    assert abs(e_sym - e_full) < 1e-12 * abs(e_full)
    assert abs(e_off - e_full) < 1e-13 * abs(e_full)


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp64", 1e-12)])
def test_full_size_reduced_equals_unreduced(prec, tol):
    """Silicon-like 4x4x4 cell, 24^3 box (8 irreducible of 64 k-points): reduced and unreduced GPU outputs
    agree on the model orbitals (a property that holds at any size)."""
    p = synth.si_params()
    S = make_setup(p)
    ops = synth.point_group(p["lattice"])
    cp, cc, eig, gap = synth.model_orbitals(p["lattice"], S.kcart, S.miller, S.npw_max, 4)
    occ = synth.occupations(S.Nk, 4, 4)
    ctx = _ctx(p, precision=prec)
    try:
        ctx.set_symmetry(ops)
        a, b = torch.from_numpy(cp).cuda(), torch.from_numpy(cc).cuda()
        ctx.symmetrize_orbitals(a, b)
        r1, l1 = ctx.apply(a, b, occ)
        r1, l1 = r1.clone(), l1.clone()
        ctx.set_symmetry([])
        r0, l0 = ctx.apply(a, b, occ)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    sc = max(float(r0.abs().max()), float(l0.abs().max()))
    assert float((r1 - r0).abs().max()) / sc < tol
    assert float((l1 - l0).abs().max()) / sc < tol


def test_symmetry_errors():
    from paper_2302_07420_gb300 import _lib
    p = synth.si_params(kmesh=(2, 2, 2), fft=9, ecut=3.0)   # spheres fit, pair densities would wrap
    ops = synth.point_group(p["lattice"])
    ctx = _ctx(p)
    try:
        with pytest.raises(_lib.TCError) as e:
            ctx.set_symmetry(ops)
        assert e.value.status == _lib.TC_ERR_UNSUPPORTED
    finally:
        ctx.close()
    p = synth.si_params(kmesh=(2, 2, 2), fft=12, ecut=1.5)
    ctx = _ctx(p)
    try:
        with pytest.raises(_lib.TCError) as e:
            ctx.set_symmetry(ops[1:])                         # identity missing
        assert e.value.status == _lib.TC_ERR_ARG
        shear = np.array([[1, 1, 0], [0, 1, 0], [0, 0, 1]])
        with pytest.raises(_lib.TCError) as e:
            ctx.set_symmetry([np.eye(3, dtype=int), shear])
        assert e.value.status == _lib.TC_ERR_ARG
        with pytest.raises(_lib.TCError) as e:
            ctx.symmetrize_orbitals(np.zeros((ctx.nk, 4, ctx.npw_max), complex),
                                    np.zeros((ctx.nk, 4, ctx.npw_max), complex))
        assert e.value.status == _lib.TC_ERR_STATE
    finally:
        ctx.close()


def test_reduced_apply_one_output_side():
    """Only the left outputs requested (right pointer null): the unfolding handles the single array."""
    import ctypes
    p, S, ops, kinfo, irred, cp, cc, up, uc = _inputs((2, 2, 2), 12, 1.5)
    occ = synth.occupations(S.Nk, 4, 4)
    ref_r, ref_l = OP.tc_apply(S, up, uc, occ)
    ctx = _ctx(p)
    try:
        ctx.set_symmetry(ops)
        a, b = torch.from_numpy(up).cuda(), torch.from_numpy(uc).cuda()
        out = torch.zeros_like(a)
        occ_np, occ_p = ctx._occ(occ)
        st = ctx.lib.tc_apply(ctx.h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), occ_p, None,
                              ctypes.c_void_p(out.data_ptr()), None)
        assert st == 0
        torch.cuda.synchronize()
    finally:
        ctx.close()
    assert np.abs(out.cpu().numpy() - ref_l).max() / np.abs(ref_l).max() < 1e-11


def test_davidson_step_with_symmetry():
    """One Davidson step on symmetric inputs with the reduction on equals the oracle's full step: Ritz
    values per k-point and the projector sum_i phi_i chi_i^H onto the new trial space (degenerate Ritz
    values at high-symmetry points make single vectors non-unique)."""
    from oracle import davidson as DV
    p, S, ops, kinfo, irred, cp, cc, up, uc = _inputs((2, 2, 2), 12, 1.5)
    occ = synth.occupations(S.Nk, 4, 4)
    phi_r, chi_r, lam_r, d_r = DV.davidson_step(S, up, uc, occ)
    ctx = _ctx(p)
    try:
        ctx.set_symmetry(ops)
        phi, chi, lam, dim = ctx.davidson_step(torch.from_numpy(up).cuda(), torch.from_numpy(uc).cuda(), occ)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    phi, chi = phi.cpu().numpy(), chi.cpu().numpy()
    np.testing.assert_array_equal(dim, d_r)
    sc = np.abs(lam_r).max()
    for k in range(S.Nk):
        assert np.abs(np.sort(lam[k].real) - np.sort(lam_r[k].real)).max() < 1e-11 * sc
        P = phi[k].T @ np.conj(chi[k])
        Pr = phi_r[k].T @ np.conj(chi_r[k])
        assert np.abs(P - Pr).max() < 1e-9
