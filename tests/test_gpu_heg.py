"""Homogeneous electron gas on the GPU against the closed forms (pin P1).

N = 114 electrons (57 plane waves |n|^2 <= 5), r_s = 2, Gamma only, 48^3 box:
every term is diagonal in momentum with the lattice-sum eigenvalues of
tests/test_oracle_heg.py (exact for the grid operator here: all products stay
far below the aliasing limit of the box), and BITC = TC (out_L = out_R).
The 48^3 work volumes do not fit in shared memory and live in global scratch.
"""
import numpy as np
import pytest

from oracle import operator as OP
from test_oracle_heg import closed_forms, heg_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _apply(S, c, occ, prec):
    from paper_2302_07420_gb300.operator import Context
    ctx = Context(S.lattice, S.kmesh, S.ecut, S.n, S.nbands, S.nocc, S.A, S.C, precision=prec)
    d = torch.from_numpy(c).cuda()
    out_r, out_l = ctx.apply(d, d, occ)
    E = ctx.energy(d, d, occ)
    ctx.close()
    return out_r.cpu().numpy(), out_l.cpu().numpy(), E


@pytest.mark.parametrize("prec,tol,etol", [("fp64", 1e-11, 1e-11), ("fp32", 1e-5, 1e-6)])
def test_heg_114_48_box_against_closed_forms(prec, tol, etol):
    S, c, occ = heg_case(nelec=114, rs=2.0, fft=48, radius2=144, radius2_occ=5)
    idx, e = closed_forms(S, c)
    eps = sum(e[t] for t in OP.TERMS)
    out_r, out_l, E = _apply(S, c, occ, prec)
    scale = np.abs(eps).max()
    diag = np.array([out_r[0, b, idx[b]] for b in range(S.nocc)])
    assert np.abs(diag - eps).max() / scale < tol
    off = out_r.copy()
    for b in range(S.nocc):
        off[0, b, idx[b]] = 0.0
    assert np.abs(off).max() / scale < tol
    assert np.abs(out_l - out_r).max() / scale < tol          # BITC = TC for plane waves
    G = S.miller[0][idx] @ S.B
    kin = 0.5 * np.einsum("ij,ij->i", G, G)
    two = sum(e[t] for t in OP.TWO_BODY)
    three = sum(e[t] for t in OP.THREE_BODY)
    Eref = float(np.real(2.0 * np.sum(kin + two / 2 + three / 3)))
    assert abs(E - Eref) / S.nocc / 2 < etol * max(1.0, abs(Eref)), (E, Eref)


_RAND48 = {}


def _random_48():
    """Random biorthonormal orbitals on a small Gamma-only cell with the 48^3 box (3 bands, 2 occupied):
    every element of the 48^3 path (global-scratch work volumes) is compared with the oracle, not only
    the diagonal plane-wave case."""
    if not _RAND48:
        from conftest import make_setup
        from paper_2302_07420_gb300 import synth
        p = synth.tiny_params(4, kmesh=(1, 1, 1), fft=(48,) * 3, ecut=2.2, nbands=3, nocc=2, scale=7.0)
        S = make_setup(p)
        c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 700, [S.kpG(0)], S.npw_max, S.nbands, perturb=0.1)
        occ = synth.occupations(1, S.nbands, S.nocc)
        occ[0, 1] = 0.6
        r, l_ = OP.tc_apply(S, c_phi, c_chi, occ)
        _RAND48.update(p=p, S=S, c_phi=c_phi, c_chi=c_chi, occ=occ, r=r, l=l_)
    return _RAND48


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_48_box_random_orbitals_against_the_oracle(prec, tol):
    from paper_2302_07420_gb300.operator import Context
    d = _random_48()
    p = d["p"]
    ctx = Context(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"],
                  precision=prec)
    try:
        a, b = torch.from_numpy(d["c_phi"]).cuda(), torch.from_numpy(d["c_chi"]).cuda()
        out_r, out_l = ctx.apply(a, b, d["occ"])
        torch.cuda.synchronize()
    finally:
        ctx.close()
    scale = max(np.abs(d["r"]).max(), np.abs(d["l"]).max())
    er = np.abs(out_r.cpu().numpy() - d["r"]).max() / scale
    el = np.abs(out_l.cpu().numpy() - d["l"]).max() / scale
    assert er < tol and el < tol, (er, el)
