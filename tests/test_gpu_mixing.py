"""Density-matrix mixing inputs (Sec. 2.4) on the GPU.

TC++ mixes density matrices by giving the operator the new orbitals with
occupations beta f and the old ones, as extra bands, with (1 - beta) f.  The
two sets are not biorthogonal to each other, which exercises the
general-overlap forms of the 3a2 corrections (Eqs.
divcor_3a2_first/second_density_matrix_mixing) and of the 3b6 corrections.
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


def _mixed(beta=0.7):
    """New and old biorthonormal sets (2 bands each) stacked as 4 partner bands plus 1 empty band."""
    p = synth.tiny_params(5, kmesh=(1, 1, 2), fft=(12,) * 3, ecut=1.6, nbands=5, nocc=4, scale=5.0)
    S = make_setup(p)
    kpg = [S.kpG(k) for k in range(S.Nk)]
    new_phi, new_chi = synth.random_orbitals(synth.SEED0 + 500, kpg, S.npw_max, 3, perturb=0.1)
    old_phi, old_chi = synth.random_orbitals(synth.SEED0 + 501, kpg, S.npw_max, 2, perturb=0.1)
    old_phi = new_phi[:, :2] + 0.05 * old_phi          # the previous loop's orbitals: close, not equal
    old_chi = new_chi[:, :2] + 0.05 * old_chi
    c_phi = np.concatenate([new_phi[:, :2], old_phi, new_phi[:, 2:]], axis=1)
    c_chi = np.concatenate([new_chi[:, :2], old_chi, new_chi[:, 2:]], axis=1)
    f = np.array([1.0, 0.8])
    occ = np.zeros((S.Nk, 5))
    occ[:, :2] = beta * f
    occ[:, 2:4] = (1.0 - beta) * f
    return p, S, c_phi, c_chi, occ


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_mixed_partner_sets_match_the_oracle(prec, tol):
    p, S, c_phi, c_chi, occ = _mixed()
    ref_r, ref_l = OP.tc_apply(S, c_phi, c_chi, occ)
    ctx = _ctx(p, precision=prec)
    out_r, out_l = ctx.apply(torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda(), occ)
    torch.cuda.synchronize()
    ctx.close()
    scale = max(np.abs(ref_r).max(), np.abs(ref_l).max())
    assert np.abs(out_r.cpu().numpy() - ref_r).max() / scale < tol
    assert np.abs(out_l.cpu().numpy() - ref_l).max() / scale < tol


def test_split_partners_give_the_unsplit_operator():
    """Two identical copies at beta f and (1 - beta) f act as one partner at f (FP64, through the C ABI)."""
    p1 = synth.tiny_params(6, kmesh=(2, 1, 1), fft=(12,) * 3, ecut=1.6, nbands=2, nocc=2, scale=5.0)
    S1 = make_setup(p1)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 502, [S1.kpG(k) for k in range(S1.Nk)], S1.npw_max, 2,
                                         perturb=0.1)
    occ1 = np.array([[1.0, 0.6]] * S1.Nk)
    ctx1 = _ctx(p1)
    r1, l1 = ctx1.apply(torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda(), occ1)
    p2 = dict(p1, nbands=4, nocc=4)
    ctx2 = _ctx(p2)
    beta = 0.35
    r2, l2 = ctx2.apply(torch.from_numpy(np.concatenate([c_phi, c_phi], axis=1)).cuda(),
                        torch.from_numpy(np.concatenate([c_chi, c_chi], axis=1)).cuda(),
                        np.concatenate([beta * occ1, (1 - beta) * occ1], axis=1))
    torch.cuda.synchronize()
    ctx1.close()
    ctx2.close()
    r1, l1, r2, l2 = (x.cpu().numpy() for x in (r1, l1, r2, l2))
    scale = np.abs(r1).max()
    for half in (slice(0, 2), slice(2, 4)):
        assert np.abs(r2[:, half] - r1).max() / scale < 1e-12
        assert np.abs(l2[:, half] - l1).max() / scale < 1e-12
