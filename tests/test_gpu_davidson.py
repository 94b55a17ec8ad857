"""tc_davidson_step against the oracle's block-Davidson step (Sec. 2.4, Appendix A).

Eigenvalues are unique and compared directly; eigenvectors are unique up to a
phase per band (the Gram-Schmidt and the biorthonormalisation carry the phase
of each Ritz vector through), so each output band is aligned to the oracle's
phase before the element-wise comparison.  Degenerate cases (plane waves of
the electron gas) compare the spans instead.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import davidson as DV
from oracle import operator as OP
from paper_2302_07420_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(p, **kw):
    from paper_2302_07420_gb300.operator import Context
    args = dict(lattice=p["lattice"], kmesh=p["kmesh"], ecut=p["ecut"], fft=p["fft"], nbands=p["nbands"],
                nocc=p["nocc"], A=p["A"], C=p["C"])
    args.update(kw)
    return Context(**args)


def _case(seed, kmesh, fft, ecut, m, nocc, perturb=0.1):
    p = synth.tiny_params(seed, kmesh=kmesh, fft=fft, ecut=ecut, nbands=m, nocc=nocc, scale=5.0)
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 700 + seed, [S.kpG(k) for k in range(S.Nk)], S.npw_max, m,
                                         perturb=perturb)
    occ = np.zeros((S.Nk, m))
    occ[:, :nocc] = np.linspace(1.0, 0.6, nocc)
    return p, S, c_phi, c_chi, occ


def _align(ref, got):
    ov = np.einsum("...i,...i->...", np.conj(ref), got)
    return got * (np.conj(ov) / np.abs(ov))[..., None]


def _run(p, c_phi, c_chi, occ, device=True, **kw):
    ctx = _ctx(p, **kw)
    try:
        if device:
            phi, chi, eig, dim = ctx.davidson_step(torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda(), occ)
            torch.cuda.synchronize()
            return phi.cpu().numpy(), chi.cpu().numpy(), eig, dim
        return ctx.davidson_step(c_phi, c_chi, occ)
    finally:
        ctx.close()


def _compare(S, ref, got, tol_eig, tol_vec):
    phi_r, chi_r, lam_r, d_r = ref
    phi_g, chi_g, lam_g, d_g = got
    np.testing.assert_array_equal(d_g, d_r)
    scale = np.abs(lam_r).max()
    assert np.abs(lam_g - lam_r).max() / scale < tol_eig
    assert np.abs(_align(phi_r, phi_g) - phi_r).max() < tol_vec
    # chi carries the phase of phi (biorthonormal pair): align with phi's phase
    ov = np.einsum("...i,...i->...", np.conj(phi_r), phi_g)
    ph = np.conj(ov) / np.abs(ov)
    assert np.abs(chi_g * ph[..., None] - chi_r).max() / np.abs(chi_r).max() < tol_vec


@pytest.mark.parametrize("seed,kmesh,fft,ecut,m,nocc", [
    (1, (1, 1, 2), (12, 12, 12), 1.6, 3, 2),      # two k-points, ragged spheres
    (2, (2, 1, 1), (15, 15, 15), 2.2, 5, 3),      # odd box, more bands than partners
    (3, (1, 1, 1), (12, 12, 12), 1.6, 4, 4),      # every band a partner
])
def test_davidson_step_matches_the_oracle_fp64(seed, kmesh, fft, ecut, m, nocc):
    p, S, c_phi, c_chi, occ = _case(seed, kmesh, fft, ecut, m, nocc)
    ref = DV.davidson_step(S, c_phi, c_chi, occ)
    got = _run(p, c_phi, c_chi, occ)
    assert np.all(got[3] == 2 * m)
    _compare(S, ref, got, 1e-11, 1e-9)


def test_davidson_step_exact_on_a_small_sphere():
    """npw <= 2 nbands: dependent new vectors are dropped and the step is the full eigen-decomposition."""
    m = 4
    p = synth.tiny_params(4, kmesh=(1, 1, 1), fft=(12, 12, 12), ecut=0.8, nbands=m, nocc=2, scale=6.0)
    S = make_setup(p)
    n = S.npw[0]
    assert m < n < 2 * m
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 710, [S.kpG(0)], S.npw_max, m, perturb=0.1)
    occ = np.zeros((1, m))
    occ[:, :2] = [1.0, 0.7]
    ref = DV.davidson_step(S, c_phi, c_chi, occ)
    got = _run(p, c_phi, c_chi, occ)
    assert got[3][0] == n
    _compare(S, ref, got, 1e-11, 1e-8)


def test_davidson_step_host_arrays_match_device_arrays():
    p, S, c_phi, c_chi, occ = _case(5, (1, 1, 2), (12, 12, 12), 1.6, 3, 2)
    dev = _run(p, c_phi, c_chi, occ, device=True)
    host = _run(p, c_phi, c_chi, occ, device=False)
    for a, b in zip(dev, host):
        np.testing.assert_allclose(np.asarray(a), np.asarray(b), rtol=0, atol=1e-13)


def test_davidson_step_fp32_operator():
    p, S, c_phi, c_chi, occ = _case(6, (1, 1, 2), (16, 16, 16), 2.0, 4, 2)
    ref = DV.davidson_step(S, c_phi, c_chi, occ)
    got = _run(p, c_phi, c_chi, occ, precision="fp32")
    _compare(S, ref, got, 2e-6, 2e-4)


def test_davidson_outputs_satisfy_appendix_a_through_the_library():
    """<phi_i|h|phi_j> from the library's own operator is upper triangular with the Ritz values on the
    diagonal (phi lies in the subspace, and Gram-Schmidt keeps the diagonal, Appendix A)."""
    p, S, c_phi, c_chi, occ = _case(7, (1, 1, 2), (12, 12, 12), 1.6, 3, 2)
    phi, chi, lam, dim = _run(p, c_phi, c_chi, occ)
    # h phi with the step's partners: partners in bands 0..nocc-1, phi in empty bands after them
    no, m = 2, 3
    pa = dict(p, nbands=no + m)
    ctx = _ctx(pa)
    bphi = np.concatenate([c_phi[:, :no], phi], axis=1)
    bchi = np.concatenate([c_chi[:, :no], phi], axis=1)
    bocc = np.concatenate([occ[:, :no], np.zeros((S.Nk, m))], axis=1)
    out, _ = ctx.apply(torch.from_numpy(bphi).cuda(), torch.from_numpy(bchi).cuda(), bocc)
    torch.cuda.synchronize()
    ctx.close()
    hphi = out.cpu().numpy()[:, no:] + OP.kinetic_coeffs(S, phi)
    for k in range(S.Nk):
        sc = np.abs(lam[k]).max()
        np.testing.assert_allclose(np.conj(phi[k]) @ phi[k].T, np.eye(m), atol=1e-12)
        np.testing.assert_allclose(np.conj(chi[k]) @ phi[k].T, np.eye(m), atol=1e-12)
        for bra in (phi[k], chi[k]):
            eps = np.conj(bra) @ hphi[k].T
            np.testing.assert_allclose(np.diag(eps), lam[k], atol=1e-11 * sc)
            assert np.abs(np.tril(eps, -1)).max() < 1e-11 * sc


@pytest.mark.parametrize("case", [dict(nelec=14, rs=4.0, fft=16, radius2=16, radius2_occ=1),
                                  dict(nelec=38, rs=2.5, fft=15, radius2=9, radius2_occ=2)])
def test_heg_plane_waves_are_fixed_points(case):
    """Degenerate shells: no new direction, the oracle's eigenvalues, the same span."""
    from test_oracle_heg import heg_case
    S, c, occ = heg_case(**case)
    p = synth.heg_params(case["nelec"], case["rs"], case["fft"], case["radius2"])
    ref = DV.davidson_step(S, c, c, occ)
    phi, chi, lam, dim = _run(p, c, c, occ)
    m = c.shape[1]
    assert dim[0] == m
    scale = np.abs(ref[2]).max()
    np.testing.assert_allclose(np.sort(lam[0].real), np.sort(ref[2][0].real), atol=1e-11 * scale)
    assert np.abs(lam[0].imag).max() < 1e-11 * scale
    np.testing.assert_allclose(phi[0].T @ np.conj(phi[0]), c[0].T @ np.conj(c[0]), atol=1e-10)
    np.testing.assert_allclose(chi[0].T @ np.conj(phi[0]), c[0].T @ np.conj(c[0]), atol=1e-10)


def test_davidson_step_rejects_aliased_outputs():
    from paper_2302_07420_gb300 import _lib
    import ctypes
    p, S, c_phi, c_chi, occ = _case(8, (1, 1, 1), (12, 12, 12), 1.6, 2, 1)
    ctx = _ctx(p)
    try:
        a = torch.from_numpy(c_phi).cuda()
        b = torch.from_numpy(c_chi).cuda()
        occ_np, occ_p = ctx._occ(occ)
        vp = ctypes.c_void_p
        st = ctx.lib.tc_davidson_step(ctx.h, vp(a.data_ptr()), vp(b.data_ptr()), occ_p, vp(a.data_ptr()),
                                      vp(b.data_ptr()), None, None, None)
        assert st == _lib.TC_ERR_ARG
    finally:
        ctx.close()


def test_davidson_step_silicon_like_2x2x2():
    """Silicon-like FCC cell, 24^3 box, 8 k-points, spheres of 254-266 plane waves (past one 256-thread
    tile, ragged), every band a partner."""
    p = synth.si_params(kmesh=(2, 2, 2))
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 720, [S.kpG(k) for k in range(S.Nk)], S.npw_max,
                                         p["nbands"], perturb=0.1)
    occ = synth.occupations(S.Nk, p["nbands"], p["nocc"])
    ref = DV.davidson_step(S, c_phi, c_chi, occ)
    got = _run(p, c_phi, c_chi, occ)
    _compare(S, ref, got, 1e-11, 1e-9)


@pytest.mark.parametrize("ecut,scale", [(4.0, 7.0), (5.0, 5.0)])
def test_davidson_step_many_bands_global_solver(ecut, scale):
    """40 bands: the subspace arrays (2 d^2 + 4 m d complex words for d up to 80) exceed shared memory,
    so the eigen-solver runs on global scratch; d = 80 (every new vector kept) and d = 59 (the sphere has
    59 plane waves: the space is exhausted and the step is exact)."""
    m = 40
    p = synth.tiny_params(11, kmesh=(1, 1, 1), fft=(18, 18, 18) if scale > 6 else (16, 16, 16), ecut=ecut,
                          nbands=m, nocc=2, scale=scale)
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 730, [S.kpG(k) for k in range(S.Nk)], S.npw_max, m,
                                         perturb=0.1)
    occ = np.zeros((S.Nk, m))
    occ[:, :2] = [1.0, 0.8]
    ref = DV.davidson_step(S, c_phi, c_chi, occ)
    got = _run(p, c_phi, c_chi, occ)
    assert got[3][0] == min(2 * m, S.npw[0])
    _compare(S, ref, got, 1e-11, 1e-8)
