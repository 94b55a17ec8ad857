"""Pair chains with pruned transforms (24^3 box) against the FP64 oracle, through the C ABI.

At 24^3 the library runs the pair chains, the 3b4 pass and the occupied-pair stage with transforms
restricted to the pair-density support (17 box indices per axis) when the Miller span s of the
spheres gives 2 s + 1 <= 17 (at 16^3 up to 13, at 18^3 and 20^3 up to 17: cases b16, b18, b20), on thread-block clusters with support 21 up to 2 s + 1 = 21, and with full
transforms beyond.  The cases cover small supports (span 2 and 6), the edge 2 s + 1 = 17 (the
silicon-like cell at 7.5 Ha, the bench cell's spheres), and a span beyond it (10 Ha, the cluster
kernels; test_gpu_cluster.py covers them and the full transforms), every term separately in FP64 and
the totals in both precisions.  Tolerances are those of the other parity tests.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import operator as OP
from paper_2302_07420_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-11, "fp32": 1e-5}


def _span(S):
    allm = np.concatenate(S.miller)
    return int((allm.max(0) - allm.min(0)).max())


def _case(name):
    if name == "tiny_span2":
        p = synth.tiny_params(9, kmesh=(1, 1, 2), fft=(24,) * 3, ecut=1.6, nbands=3, nocc=2, scale=5.0)
    elif name == "tiny_span6":
        p = synth.tiny_params(11, kmesh=(1, 1, 2), fft=(24,) * 3, ecut=6.0, nbands=3, nocc=2, scale=5.0)
    elif name == "b16_span6":
        p = synth.tiny_params(31, kmesh=(1, 1, 2), fft=(16,) * 3, ecut=6.0, nbands=3, nocc=2, scale=5.0)
    elif name == "b18_span8":
        p = synth.tiny_params(32, kmesh=(2, 1, 1), fft=(18,) * 3, ecut=10.0, nbands=3, nocc=2, scale=5.0)
    elif name == "b20_span6":
        p = synth.tiny_params(33, kmesh=(1, 2, 1), fft=(20,) * 3, ecut=10.0, nbands=3, nocc=2, scale=5.0)
    elif name == "si_k112_edge":
        p = synth.si_params(kmesh=(1, 1, 2), nbands=3, nocc=2)
    else:   # "si_k112_wide": span 10, beyond the one-CTA pruned support
        p = synth.si_params(kmesh=(1, 1, 2), ecut=10.0, nbands=3, nocc=2)
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 400 + len(name), [S.kpG(k) for k in range(S.Nk)],
                                         S.npw_max, S.nbands, perturb=0.1)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, : S.nocc] = np.array([1.0, 0.6])[None]
    return p, S, c_phi, c_chi, occ


EXPECTED_SPAN = {"tiny_span2": 2, "tiny_span6": 6, "si_k112_edge": 8, "si_k112_wide": 10, "b16_span6": 6,
                 "b18_span8": 8, "b20_span6": 6}
_REF = {}


def _ref(name):
    if name not in _REF:
        p, S, c_phi, c_chi, occ = _case(name)
        assert _span(S) == EXPECTED_SPAN[name]
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


@pytest.mark.parametrize("name", ["tiny_span6", "si_k112_edge", "b16_span6", "b18_span8", "b20_span6"])
def test_pruned_chain_every_term_fp64(name):
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref(name)
    scale = max(np.abs(OP.total(ref_r)).max(), np.abs(OP.total(ref_l)).max())
    for t_i, t in enumerate(OP.TERMS):
        ctx = _ctx(p, term_mask=1 << t_i)
        out_r, out_l = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
        torch.cuda.synchronize()
        er = np.abs(out_r.cpu().numpy() - ref_r[t]).max() / scale
        el = np.abs(out_l.cpu().numpy() - ref_l[t]).max() / scale
        ctx.close()
        assert er < TOL["fp64"] and el < TOL["fp64"], (t, er, el)


@pytest.mark.parametrize("name", ["tiny_span2", "tiny_span6", "si_k112_edge", "si_k112_wide", "b16_span6",
                                  "b18_span8", "b20_span6"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pruned_chain_total(name, prec):
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref(name)
    tr, tl = OP.total(ref_r), OP.total(ref_l)
    scale = max(np.abs(tr).max(), np.abs(tl).max())
    ctx = _ctx(p, precision=prec)
    if name.startswith("b") or name in ("tiny_span2", "tiny_span6", "si_k112_edge"):
        assert all(v[0] == 1 for v in ctx.pair_kernels().values()), ctx.pair_kernels()
    out_r, out_l = ctx.apply(_dev(c_phi), _dev(c_chi), occ)
    torch.cuda.synchronize()
    er = np.abs(out_r.cpu().numpy() - tr).max() / scale
    el = np.abs(out_l.cpu().numpy() - tl).max() / scale
    ctx.close()
    assert er < TOL[prec] and el < TOL[prec], (er, el)


def test_pruned_chain_chunked_and_one_sided_energy():
    """Partner chunks (autotuned counts) and the one-sided energy launch take the same pruned kernels."""
    p, S, c_phi, c_chi, occ, ref_r, ref_l = _ref("si_k112_edge")
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
