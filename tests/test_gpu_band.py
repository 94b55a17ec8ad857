"""Band-structure k-points off the SCF mesh on the GPU (tc_init_band / tc_apply_band) against the
band-point oracle (oracle/band.py), through the C ABI.

Sec. 2.6.3 after Eq. divcorr_2ax_scf and Sec. 2.6.4: outputs at band points k_b, partners on the SCF
mesh, kernels at k_b - q + G, the band forms of the divergence corrections (Gamma_b, W(k_b)) with the
band point's own occupied orbitals.  Cases: tiny triclinic cells (one and two band points, 9^3 and
12^3 boxes, partial occupations, corrections on and off), every term separately in FP64 (1e-11) and
the totals in FP64 and FP32 (1e-5); the full-size silicon-like 4x4x4 cell at one band point against
the stored oracle values (tests/golden/si_k444_band.json).
"""
import json
import os
import sys

import numpy as np
import pytest

from conftest import make_setup
from oracle import band as BD
from oracle import operator as OP
from paper_2302_07420_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {"fp64": 1e-11, "fp32": 1e-5}
K_OFF = ((0.13, 0.27, -0.31),)
K_TWO = ((0.13, 0.27, -0.31), (0.5, 0.0, 0.125))


def _case(seed, kmesh, fft, kfrac, div=1, ecut=1.6):
    p = synth.tiny_params(seed, kmesh=kmesh, fft=(fft,) * 3, ecut=ecut, nbands=3, nocc=2, scale=5.0)
    S = make_setup(p, div_correction=div)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 60 + seed, [S.kpG(k) for k in range(S.Nk)], S.npw_max,
                                         S.nbands, perturb=0.2)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, 1] = 0.6
    SB = BD.BandSetup(S, kfrac)
    kp = [SB.kpG(S.Nk + i) for i in range(SB.nkb)]
    b_phi, b_chi = synth.random_orbitals(synth.SEED0 + 80 + seed, kp, SB.npw_max, S.nbands, perturb=0.2)
    b_occ = synth.occupations(SB.nkb, S.nbands, S.nocc)
    b_occ[:, 1] = 0.7
    p = dict(p, div_correction=div)
    return p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ


def _pad(c, n):
    out = np.zeros(c.shape[:-1] + (n,), dtype=np.complex128)
    out[..., : c.shape[-1]] = c
    return out


def _ctx(p, kfrac, **kw):
    from paper_2302_07420_gb300.operator import BandContext
    args = dict(lattice=p["lattice"], kmesh=p["kmesh"], ecut=p["ecut"], fft=p["fft"], nbands=p["nbands"],
                nocc=p["nocc"], A=p["A"], C=p["C"], div_correction=p.get("div_correction", 1))
    args.update(kw)
    return BandContext(kfrac_band=kfrac, **args)


def _run(ctx, c_phi, c_chi, occ, b_phi, b_chi, b_occ):
    n = ctx.npw_max
    d = [torch.from_numpy(_pad(x, n)).cuda() for x in (c_phi, c_chi, b_phi, b_chi)]
    r, l = ctx.apply_band(d[0], d[1], occ, d[2], d[3], b_occ)
    torch.cuda.synchronize()
    return r.cpu().numpy(), l.cpu().numpy()


CASES = [(1, (1, 1, 2), 9, K_OFF, 1), (2, (2, 1, 1), 12, K_TWO, 1), (3, (1, 2, 1), 9, K_OFF, 0)]
_REF = {}


def _ref(case):
    if case not in _REF:
        seed, kmesh, fft, kfrac, div = case
        p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ = _case(seed, kmesh, fft, kfrac, div)
        r = BD.band_apply(S, c_phi, c_chi, occ, kfrac, b_phi, b_chi, b_occ, left=False)
        l_ = BD.band_apply(S, c_phi, c_chi, occ, kfrac, b_phi, b_chi, b_occ, left=True)
        _REF[case] = (p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ, r, l_)
    return _REF[case]


def test_band_layout_matches_the_oracle():
    p, S, SB, *_ = _ref(CASES[1])
    ctx = _ctx(p, K_TWO)
    try:
        npw, miller = ctx.layout()
        assert ctx.nk == S.Nk + 2 and ctx.npw_max == SB.npw_max
        for k in range(ctx.nk):
            assert npw[k] == SB.npw[k]
            assert np.array_equal(miller[k, : npw[k]], SB.miller[k])
    finally:
        ctx.close()


@pytest.mark.parametrize("case", CASES[:2], ids=["k112_9_one_point", "k211_12_two_points"])
def test_band_every_term_fp64(case):
    p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ, ref_r, ref_l = _ref(case)
    kfrac = case[3]
    scale = max(np.abs(OP.total(ref_r)).max(), np.abs(OP.total(ref_l)).max())
    for t_i, t in enumerate(OP.TERMS):
        ctx = _ctx(p, kfrac, term_mask=1 << t_i)
        try:
            out_r, out_l = _run(ctx, c_phi, c_chi, occ, b_phi, b_chi, b_occ)
        finally:
            ctx.close()
        n = SB.npw_max
        er = np.abs(out_r[..., :n] - ref_r[t]).max() / scale
        el = np.abs(out_l[..., :n] - ref_l[t]).max() / scale
        assert er < TOL["fp64"] and el < TOL["fp64"], (t, er, el)


@pytest.mark.parametrize("case", CASES, ids=["k112_9_one_point", "k211_12_two_points", "k121_9_no_corrections"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_band_total(case, prec):
    p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ, ref_r, ref_l = _ref(case)
    tr, tl = OP.total(ref_r), OP.total(ref_l)
    scale = max(np.abs(tr).max(), np.abs(tl).max())
    ctx = _ctx(p, case[3], precision=prec)
    try:
        out_r, out_l = _run(ctx, c_phi, c_chi, occ, b_phi, b_chi, b_occ)
    finally:
        ctx.close()
    n = SB.npw_max
    er = np.abs(out_r[..., :n] - tr).max() / scale
    el = np.abs(out_l[..., :n] - tl).max() / scale
    assert er < TOL[prec] and el < TOL[prec], (er, el)


def test_band_context_refuses_mesh_points_and_mesh_calls():
    from paper_2302_07420_gb300 import _lib
    p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ, *_ = _ref(CASES[0])
    with pytest.raises(_lib.TCError) as e:
        _ctx(p, [[0.0, 0.0, 0.5]])             # the mesh point (0, 0, 1/2) of the 1x1x2 mesh
    assert e.value.status == _lib.TC_ERR_ARG
    ctx = _ctx(p, K_OFF)
    try:
        x = torch.zeros((ctx.nk, ctx.nbands, ctx.npw_max), dtype=torch.complex128, device="cuda")
        with pytest.raises(_lib.TCError) as e:
            ctx.apply(x, x, np.ones((ctx.nk, ctx.nbands)))
        assert e.value.status == _lib.TC_ERR_STATE
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_band_si_k444_against_the_stored_oracle_values(prec):
    """Full size: the 4x4x4 silicon-like cell (24^3 box) with one band point, against
    tests/golden/si_k444_band.json (oracle only, make_golden.py)."""
    path = os.path.join(HERE, "golden", "si_k444_band.json")
    g = json.load(open(path))
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden as MG
    p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ = MG.band_inputs()
    ctx = _ctx(p, [g["k_band_frac"]], precision=prec)
    try:
        out_r, out_l = _run(ctx, c_phi, c_chi, occ, b_phi, b_chi, b_occ)
    finally:
        ctx.close()
    npw = g["npw_band"]
    ref_r = np.array(g["out_R"]).view(complex).reshape(S.nbands, npw)
    ref_l = np.array(g["out_L"]).view(complex).reshape(S.nbands, npw)
    scale = max(np.abs(ref_r).max(), np.abs(ref_l).max())
    er = np.abs(out_r[0, :, :npw] - ref_r).max() / scale
    el = np.abs(out_l[0, :, :npw] - ref_l).max() / scale
    assert er < TOL[prec] and el < TOL[prec], (er, el)
