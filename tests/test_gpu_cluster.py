"""Pair kernels on thread-block clusters (24^3 .. 48^3 boxes) against the FP64 oracle, through the C ABI.

For boxes whose pruned volumes do not fit one CTA's shared memory, the pair chains, the 3b4 pass and the
occupied-pair stage split each item over a thread-block cluster (tc_pair_kernels kind 2) when the
pair-density support 2 s + 1 (s: Miller span of the spheres) fits the support compiled for the box: 21 at
24^3 (above the 17 of the one-CTA pruned kernels), 25 at 25^3 and 27^3, 29 at 30^3 and 32^3, and the full
box at 48^3.  Beyond the compiled support the one-CTA
kernels with full transforms run (kind 0).  Cases: spans
from 2 to 11 on triclinic and silicon-like cells, 1-2 k-points, partial occupations; every term
separately in FP64 (1e-11) and the totals in FP64 and FP32 (1e-5); partner chunks and the one-sided
energy; a band point off the mesh; the symmetry-reduced occupied-pair stage; the one-CTA fallback
when no cluster fits the device (forced by the host fault switch TC_FAULT=nocluster).
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import band as BD
from oracle import operator as OP
from oracle import symmetry as SY
from paper_2302_07420_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-11, "fp32": 1e-5}


def _span(S):
    allm = np.concatenate(S.miller)
    return int((allm.max(0) - allm.min(0)).max())


# name: (params, expected span, expected kinds of the pair-chain, 3b4 and occupied-pair kernels in FP32)
CASES = {
    "c25_span8": (lambda: synth.tiny_params(21, kmesh=(1, 1, 2), fft=(25,) * 3, ecut=12.0, nbands=3, nocc=2,
                                            scale=5.0), 8, (2, 2, 2)),
    "c27_span5": (lambda: synth.tiny_params(22, kmesh=(2, 1, 1), fft=(27,) * 3, ecut=6.0, nbands=3, nocc=2,
                                            scale=5.0), 5, (2, 2, 2)),
    "c30_span4": (lambda: synth.tiny_params(23, kmesh=(1, 2, 1), fft=(30,) * 3, ecut=4.0, nbands=3, nocc=2,
                                            scale=5.0), 4, (2, 2, 2)),
    "c32_span8": (lambda: synth.tiny_params(24, kmesh=(1, 1, 2), fft=(32,) * 3, ecut=10.0, nbands=3, nocc=2,
                                            scale=5.0), 8, (2, 2, 2)),
    "c48_span4": (lambda: synth.tiny_params(25, kmesh=(1, 1, 1), fft=(48,) * 3, ecut=3.0, nbands=3, nocc=2,
                                            scale=5.0), 4, (2, 2, 2)),
    "c24_span10": (lambda: synth.si_params(kmesh=(1, 1, 2), ecut=10.0, nbands=3, nocc=2), 10, (2, 2, 2)),
    "f24_span11": (lambda: synth.si_params(kmesh=(1, 1, 2), ecut=12.0, nbands=3, nocc=2), 11, (0, 0, 0)),
    "f27_span13": (lambda: synth.si_params(kmesh=(1, 1, 2), fft=27, ecut=16.0, nbands=3, nocc=2), 13, (0, 0, 0)),
}
_REF = {}


def _ref(name):
    if name not in _REF:
        make, span, _ = CASES[name]
        p = make()
        S = make_setup(p)
        assert _span(S) == span
        c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 500 + len(name), [S.kpG(k) for k in range(S.Nk)],
                                             S.npw_max, S.nbands, perturb=0.1)
        occ = synth.occupations(S.Nk, S.nbands, S.nocc)
        occ[:, : S.nocc] = np.array([1.0, 0.6])[None]
        r = OP.apply_operator(S, c_phi, c_chi, occ, left=False)
        l_ = OP.apply_operator(S, c_phi, c_chi, occ, left=True)
        _REF[name] = (p, S, c_phi, c_chi, occ, r, l_)
    return _REF[name]


def _ctx(p, **kw):
    from paper_2302_07420_gb300.operator import Context
    args = dict(lattice=p["lattice"], kmesh=p["kmesh"], ecut=p["ecut"], fft=p["fft"], nbands=p["nbands"],
                nocc=p["nocc"], A=p["A"], C=p["C"])
    args.update(kw)
    return Context(**args)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _kinds(ctx):
    return {k: v[0] for k, v in ctx.pair_kernels().items()}


@pytest.mark.parametrize("name", ["c25_span8", "c32_span8", "c48_span4", "f24_span11"])
def test_cluster_every_term_fp64(name):
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref(name)
    scale = max(np.abs(OP.total(ref_r)).max(), np.abs(OP.total(ref_l)).max())
    for t_i, t in enumerate(OP.TERMS):
        ctx = _ctx(p, term_mask=1 << t_i)
        try:
            out_r, out_l = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
            torch.cuda.synchronize()
        finally:
            ctx.close()
        er = np.abs(out_r.cpu().numpy() - ref_r[t]).max() / scale
        el = np.abs(out_l.cpu().numpy() - ref_l[t]).max() / scale
        assert er < TOL["fp64"] and el < TOL["fp64"], (t, er, el)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cluster_total(name, prec):
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref(name)
    tr, tl = OP.total(ref_r), OP.total(ref_l)
    scale = max(np.abs(tr).max(), np.abs(tl).max())
    ctx = _ctx(p, precision=prec)
    try:
        kinds = _kinds(ctx)
        out_r, out_l = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    if prec == "fp32":
        assert (kinds["pair_chain"], kinds["pair_3b4"], kinds["occ_pairs"]) == CASES[name][2], kinds
    er = np.abs(out_r.cpu().numpy() - tr).max() / scale
    el = np.abs(out_l.cpu().numpy() - tl).max() / scale
    assert er < TOL[prec] and el < TOL[prec], (er, el)


def test_cluster_plan_is_reported():
    """tc_pair_kernels: the one-CTA pruned kernels at 24^3 for spans up to 8, clusters for the three
    pair kernels at 32^3 in FP32 (2, 2 and 3 CTAs), full transforms beyond the compiled support."""
    p, *_ = _ref("c32_span8")
    ctx = _ctx(p, precision="fp32")
    try:
        info = ctx.pair_kernels()
    finally:
        ctx.close()
    assert info == {"pair_chain": (2, 29, 2), "pair_3b4": (2, 29, 2), "occ_pairs": (2, 29, 3)}, info
    p = synth.si_params(kmesh=(1, 1, 2), nbands=3, nocc=2)      # span 8 at 24^3
    ctx = _ctx(p, precision="fp32")
    try:
        info = ctx.pair_kernels()
    finally:
        ctx.close()
    assert info == {k: (1, 17, 1) for k in ("pair_chain", "pair_3b4", "occ_pairs")}, info
    p, *_ = _ref("f27_span13")
    ctx = _ctx(p, precision="fp32")
    try:
        info = ctx.pair_kernels()
    finally:
        ctx.close()
    assert info == {k: (0, 27, 1) for k in ("pair_chain", "pair_3b4", "occ_pairs")}, info


@pytest.mark.parametrize("name", ["c25_span8", "c32_span8", "c48_span4"])
def test_one_cta_fallback_when_no_cluster_fits(name, monkeypatch):
    """TC_FAULT=nocluster (a device that cannot hold the clusters): the contexts take the one-CTA kernels
    with full transforms, reported by tc_pair_kernels, and compute the same operator."""
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref(name)
    tr, tl = OP.total(ref_r), OP.total(ref_l)
    scale = max(np.abs(tr).max(), np.abs(tl).max())
    monkeypatch.setenv("TC_FAULT", "nocluster")
    for prec in ("fp64", "fp32"):
        ctx = _ctx(p, precision=prec)
        try:
            info = ctx.pair_kernels()
            out_r, out_l = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
            torch.cuda.synchronize()
        finally:
            ctx.close()
        assert info == {k: (0, p["fft"][0], 1) for k in ("pair_chain", "pair_3b4", "occ_pairs")}, info
        er = np.abs(out_r.cpu().numpy() - tr).max() / scale
        el = np.abs(out_l.cpu().numpy() - tl).max() / scale
        assert er < TOL[prec] and el < TOL[prec], (prec, er, el)


def test_cluster_chunked_and_one_sided_energy():
    """Partner chunks (autotuned counts) and the one-sided energy launch take the same cluster kernels."""
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref("c32_span8")
    ref_e = OP.energy_terms(S, c_phi, c_chi, occ, res=ref_r)
    ctx = _ctx(p)
    try:
        ctx.autotune(_dev(c_phi), _dev(c_chi), occ)
        out_r, out_l = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
        E = ctx.energy(_dev(c_phi), _dev(c_chi), occ)
    finally:
        ctx.close()
    tr, tl = OP.total(ref_r), OP.total(ref_l)
    scale = max(np.abs(tr).max(), np.abs(tl).max())
    assert np.abs(out_r.cpu().numpy() - tr).max() / scale < TOL["fp64"]
    assert np.abs(out_l.cpu().numpy() - tl).max() / scale < TOL["fp64"]
    assert abs(E - ref_e["total"]) < 1e-12 * max(abs(v) for v in ref_e.values())


def _pad(c, n):
    out = np.zeros(c.shape[:-1] + (n,), dtype=np.complex128)
    out[..., : c.shape[-1]] = c
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cluster_band_point(prec):
    """A band point off the mesh on a 25^3 box: the band point's own occupied-pair launch and its output
    chains run on clusters."""
    from paper_2302_07420_gb300.operator import BandContext
    kfrac = ((0.13, 0.27, -0.31),)
    p = synth.tiny_params(26, kmesh=(1, 1, 2), fft=(25,) * 3, ecut=4.0, nbands=3, nocc=2, scale=5.0)
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 560, [S.kpG(k) for k in range(S.Nk)], S.npw_max, S.nbands,
                                         perturb=0.2)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, 1] = 0.6
    SB = BD.BandSetup(S, kfrac)
    kp = [SB.kpG(S.Nk + i) for i in range(SB.nkb)]
    b_phi, b_chi = synth.random_orbitals(synth.SEED0 + 561, kp, SB.npw_max, S.nbands, perturb=0.2)
    b_occ = synth.occupations(SB.nkb, S.nbands, S.nocc)
    b_occ[:, 1] = 0.7
    ref_r = OP.total(BD.band_apply(S, c_phi, c_chi, occ, kfrac, b_phi, b_chi, b_occ, left=False))
    ref_l = OP.total(BD.band_apply(S, c_phi, c_chi, occ, kfrac, b_phi, b_chi, b_occ, left=True))
    ctx = BandContext(kfrac_band=kfrac, lattice=p["lattice"], kmesh=p["kmesh"], ecut=p["ecut"], fft=p["fft"],
                      nbands=p["nbands"], nocc=p["nocc"], A=p["A"], C=p["C"], precision=prec)
    try:
        assert _kinds(ctx)["pair_chain"] == 2
        n = ctx.npw_max
        d = [torch.from_numpy(_pad(x, n)).cuda() for x in (c_phi, c_chi, b_phi, b_chi)]
        r, l_ = ctx.apply_band(d[0], d[1], occ, d[2], d[3], b_occ)
        torch.cuda.synchronize()
        r, l_ = r.cpu().numpy(), l_.cpu().numpy()
    finally:
        ctx.close()
    scale = max(np.abs(ref_r).max(), np.abs(ref_l).max())
    m = SB.npw_max
    er = np.abs(r[..., :m] - ref_r).max() / scale
    el = np.abs(l_[..., :m] - ref_l).max() / scale
    assert er < TOL[prec] and el < TOL[prec], (er, el)


def test_cluster_symmetry_reduced():
    """Symmetry-reduced occupied-pair stage and output chains of the irreducible k-points on a 25^3 box
    (silicon-like cell, 2x2x2 mesh, model orbitals with the diamond point group) against the full oracle."""
    p = synth.si_params(kmesh=(2, 2, 2), fft=25, ecut=1.5)
    S = make_setup(p)
    ops = synth.point_group(p["lattice"])
    kinfo, irred = SY.kmap(ops, S.kfrac, True)
    cp, cc, eig, gap = synth.model_orbitals(p["lattice"], S.kcart, S.miller, S.npw_max, 4)
    assert gap > 0.05
    up = SY.unfold_orbitals(S, cp, ops, kinfo)
    uc = SY.unfold_orbitals(S, cc, ops, kinfo)
    occ = synth.occupations(S.Nk, 4, 4)
    ref_r, ref_l = OP.tc_apply(S, up, uc, occ)
    ctx = _ctx(p)
    try:
        assert _kinds(ctx)["pair_chain"] == 2
        ctx.set_symmetry(ops)
        r, l_ = ctx.apply(torch.from_numpy(up).cuda(), torch.from_numpy(uc).cuda(), occ)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    sc = max(np.abs(ref_r).max(), np.abs(ref_l).max())
    assert np.abs(r.cpu().numpy() - ref_r).max() / sc < TOL["fp64"]
    assert np.abs(l_.cpu().numpy() - ref_l).max() / sc < TOL["fp64"]
