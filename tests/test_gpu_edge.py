"""Degenerate and edge cases of the operator on the GPU against the oracle.

* Hartree-Fock limit (A = 0): every Jastrow kernel vanishes and only 2ah and 2ax remain (the TC
  operator reduces to Hartree plus exchange, Sec. 2.2).
* No occupied weight (every f = 0): every term and every divergence correction is zero.
* The smallest problem: one k-point and one band (one orbital pair per side), and one occupied of two.
* An explicit alpha of the auxiliary function (Eq. correction2): the outputs follow the oracle at that
  alpha and do not depend on it.
"""
import numpy as np
import pytest

from conftest import make_setup
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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _case(seed, kmesh, fft, nbands=3, nocc=2, **setup_kw):
    p = synth.tiny_params(seed, kmesh=kmesh, fft=(fft,) * 3, ecut=1.6, nbands=nbands, nocc=nocc, scale=5.0)
    S = make_setup(p, **setup_kw)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 300 + seed, [S.kpG(k) for k in range(S.Nk)], S.npw_max,
                                         S.nbands, perturb=0.1)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    return p, S, c_phi, c_chi, occ


def _run(p, c_phi, c_chi, occ, **kw):
    ctx = _ctx(p, **kw)
    try:
        r, l = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
        torch.cuda.synchronize()
        return r.cpu().numpy(), l.cpu().numpy()
    finally:
        ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_hartree_fock_limit(prec, tol):
    A0 = [0.0, 0.0]
    p, S, c_phi, c_chi, occ = _case(4, (1, 1, 2), 12, A=A0)
    occ[:, 1] = 0.7
    terms = OP.apply_operator(S, c_phi, c_chi, occ)
    for t in OP.TERMS:
        if t not in ("2ah", "2ax"):
            assert np.abs(terms[t]).max() == 0.0, t
    ref_r, ref_l = OP.tc_apply(S, c_phi, c_chi, occ)
    r, l = _run(p, c_phi, c_chi, occ, A=A0, precision=prec)
    sc = max(np.abs(ref_r).max(), np.abs(ref_l).max())
    assert np.abs(r - ref_r).max() / sc < tol
    assert np.abs(l - ref_l).max() / sc < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_no_occupied_weight_gives_zero(prec):
    p, S, c_phi, c_chi, occ = _case(5, (2, 1, 1), 12)
    occ[:] = 0.0
    ref_r, ref_l = OP.tc_apply(S, c_phi, c_chi, occ)
    assert np.abs(ref_r).max() == 0.0 and np.abs(ref_l).max() == 0.0
    r, l = _run(p, c_phi, c_chi, occ, precision=prec)
    assert np.abs(r).max() == 0.0 and np.abs(l).max() == 0.0


@pytest.mark.parametrize("nbands,nocc", [(1, 1), (2, 1)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_one_kpoint_one_occupied_band(nbands, nocc, prec, tol):
    p, S, c_phi, c_chi, occ = _case(6, (1, 1, 1), 9, nbands=nbands, nocc=nocc)
    ref_r, ref_l = OP.tc_apply(S, c_phi, c_chi, occ)
    r, l = _run(p, c_phi, c_chi, occ, precision=prec)
    sc = max(np.abs(ref_r).max(), np.abs(ref_l).max())
    assert np.abs(r - ref_r).max() / sc < tol
    assert np.abs(l - ref_l).max() / sc < tol


def test_explicit_alpha():
    from oracle import cell as CL
    p, S0, c_phi, c_chi, occ = _case(7, (1, 2, 1), 12)
    a = (CL.shortest_supercell_vector(p["lattice"], p["kmesh"]) / 15.0) ** 2
    S = make_setup(p, alpha=a)
    assert abs(S.alpha - a) < 1e-15 * a and abs(S.alpha - S0.alpha) > 0.1 * a
    ref_r, ref_l = OP.tc_apply(S, c_phi, c_chi, occ)
    r, l = _run(p, c_phi, c_chi, occ, alpha=a, precision="fp64")
    r0, l0 = _run(p, c_phi, c_chi, occ, precision="fp64")
    sc = max(np.abs(ref_r).max(), np.abs(ref_l).max())
    assert np.abs(r - ref_r).max() / sc < 1e-11 and np.abs(l - ref_l).max() / sc < 1e-11
    assert np.abs(r - r0).max() / sc < 1e-10 and np.abs(l - l0).max() / sc < 1e-10
