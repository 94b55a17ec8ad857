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
