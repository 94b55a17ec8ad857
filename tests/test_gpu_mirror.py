"""Mirrored two-sided pair chains against the FP64 oracle and against unmirrored applies, through the C ABI.

A two-sided FP64 apply whose pair chains run the pruned kernels computes the right side first and stores,
for every pair whose output band is itself a partner, the conjugate reflections of its pair spectrum
and of its antiparallel 3b6 spectrum; the left pair chains of the mirrored pairs take them instead of
computing their own (the left pair density of output q and partner j is the complex conjugate of the
right one of output j and partner q, Eq. BITCSCFconj; u~ is real and even, Appendix B).  The cases:
more bands than partners (band 2 has no mirror), every band a partner, a partner band with zero
occupation (its left pairs compute their own spectra), every term separately, the totals, and the
same applies with the buffer withheld (TC_FAULT=nomirror), which must agree to rounding.  FP32
contexts hold no buffer (their pair chains are bound by the loads both sides keep).  Tolerances are
those of the other parity tests.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import operator as OP
from paper_2302_07420_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-11, "fp32": 1e-5}


def _case(name):
    if name == "si_k112_nb3":
        p = synth.si_params(kmesh=(1, 1, 2), nbands=3, nocc=2)
        occ_occ = [1.0, 0.6]
    elif name == "si_k112_nb2":
        p = synth.si_params(kmesh=(1, 1, 2), nbands=2, nocc=2)
        occ_occ = [0.9, 0.7]
    elif name == "si_k112_zero":
        p = synth.si_params(kmesh=(1, 1, 2), nbands=3, nocc=3)
        occ_occ = [1.0, 0.0, 0.5]
    else:   # "b16_nb3": the 16^3 pruned kernels (support 13)
        p = synth.tiny_params(31, kmesh=(1, 1, 2), fft=(16,) * 3, ecut=6.0, nbands=3, nocc=2, scale=5.0)
        occ_occ = [1.0, 0.6]
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 700 + len(name), [S.kpG(k) for k in range(S.Nk)],
                                         S.npw_max, S.nbands, perturb=0.1)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, : S.nocc] = np.array(occ_occ)[None]
    return p, S, c_phi, c_chi, occ


_REF = {}


def _ref(name):
    if name not in _REF:
        p, S, c_phi, c_chi, occ = _case(name)
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


def _apply(p, c_phi, c_chi, occ, **kw):
    ctx = _ctx(p, **kw)
    try:
        mirror = ctx.pair_mirror()
        kinds = ctx.pair_kernels()
        out_r, out_l = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
        torch.cuda.synchronize()
        return out_r.cpu().numpy(), out_l.cpu().numpy(), mirror, kinds
    finally:
        ctx.close()


@pytest.mark.parametrize("name", ["si_k112_nb3", "si_k112_nb2", "si_k112_zero", "b16_nb3"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mirrored_total(name, prec):
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref(name)
    tr, tl = OP.total(ref_r), OP.total(ref_l)
    scale = max(np.abs(tr).max(), np.abs(tl).max())
    out_r, out_l, (active, nbytes), kinds = _apply(p, c_phi, c_chi, occ, precision=prec)
    assert kinds["pair_chain"][0] == 1, kinds
    L = kinds["pair_chain"][1]
    M = S.Nk * S.nocc
    if prec == "fp64":
        assert active and nbytes == M * M * 2 * L ** 3 * 16
    else:
        assert not active and nbytes == 0
    er = np.abs(out_r - tr).max() / scale
    el = np.abs(out_l - tl).max() / scale
    assert er < TOL[prec] and el < TOL[prec], (er, el)


@pytest.mark.parametrize("name", ["si_k112_nb3", "si_k112_zero"])
def test_mirrored_every_term_fp64(name):
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref(name)
    scale = max(np.abs(OP.total(ref_r)).max(), np.abs(OP.total(ref_l)).max())
    for t_i, t in enumerate(OP.TERMS):
        out_r, out_l, (active, _), _k = _apply(p, c_phi, c_chi, occ, term_mask=1 << t_i)
        assert active
        er = np.abs(out_r - ref_r[t]).max() / scale
        el = np.abs(out_l - ref_l[t]).max() / scale
        assert er < TOL["fp64"] and el < TOL["fp64"], (t, er, el)


def test_mirrored_equals_unmirrored(monkeypatch):
    """The same apply with the reflection buffer withheld (each side computes its own spectra): the
    right side is the same computation, the left one equal to rounding."""
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref("si_k112_nb3")
    a_r, a_l, (on, _), _k = _apply(p, c_phi, c_chi, occ)
    monkeypatch.setenv("TC_FAULT", "nomirror")
    b_r, b_l, (off, nbytes), _k = _apply(p, c_phi, c_chi, occ)
    assert on and not off and nbytes == 0
    scale = max(np.abs(a_r).max(), np.abs(a_l).max())
    assert np.array_equal(a_r, b_r)
    assert np.abs(a_l - b_l).max() / scale < 1e-13


def test_mirror_chunked_and_one_sided_energy():
    """Autotuned partner chunks on the mirrored launches, then a one-sided energy (no mirror)."""
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref("si_k112_nb3")
    ref_e = OP.energy_terms(S, c_phi, c_chi, occ, res=ref_r)
    ctx = _ctx(p)
    try:
        assert ctx.pair_mirror()[0]
        ctx.autotune(_dev(c_phi), _dev(c_chi), occ)
        out_r, out_l = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
        E = ctx.energy(_dev(c_phi), _dev(c_chi), occ)
        out_r2, out_l2 = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
    finally:
        ctx.close()
    tr, tl = OP.total(ref_r), OP.total(ref_l)
    scale = max(np.abs(tr).max(), np.abs(tl).max())
    for o_r, o_l in ((out_r, out_l), (out_r2, out_l2)):
        assert np.abs(o_r.cpu().numpy() - tr).max() / scale < TOL["fp64"]
        assert np.abs(o_l.cpu().numpy() - tl).max() / scale < TOL["fp64"]
    assert abs(E - ref_e["total"]) < 1e-12 * max(abs(v) for v in ref_e.values())


def test_no_mirror_without_pruned_kernels():
    """Contexts whose pair chains do not run the pruned kernels hold no buffer."""
    p = synth.si_params(kmesh=(1, 1, 2), ecut=10.0, nbands=3, nocc=2)   # support beyond the pruned kernels
    ctx = _ctx(p)
    try:
        assert ctx.pair_kernels()["pair_chain"][0] != 1
        assert ctx.pair_mirror() == (False, 0)
    finally:
        ctx.close()
