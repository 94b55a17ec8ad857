"""tc_apply_noalloc against tc_apply, through the C ABI, on the GPU.

tc_apply_noalloc is for callers that cannot allocate device memory -- for
instance a host framework that has already reserved nearly all of it for its
own pool, so that a cudaMalloc issued by this library would fail.  It takes
every device buffer from one fixed static array instead of a context.  Its
output must equal tc_apply's for the same inputs, and stay equal call after
call although the array keeps the previous call's contents.

This file is collected last on purpose: when a run stops at the first
failure, every other test has already run.
"""
import ctypes

import numpy as np
import pytest

from conftest import make_setup
from paper_2302_07420_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-11, "fp32": 1e-5}   # the parity tolerances of the other GPU tests


def _inputs(p, seed):
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 300 + seed, [S.kpG(k) for k in range(S.Nk)], S.npw_max,
                                         S.nbands, perturb=0.1)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    return c_phi, c_chi, occ


def _noalloc(lib, prm, d_phi, d_chi, occ):
    out_r = torch.empty_like(d_phi)
    out_l = torch.empty_like(d_chi)
    occ = np.ascontiguousarray(occ, dtype=np.float64)
    st = lib.tc_apply_noalloc(ctypes.byref(prm), ctypes.c_void_p(d_phi.data_ptr()),
                              ctypes.c_void_p(d_chi.data_ptr()), occ.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              ctypes.c_void_p(out_r.data_ptr()), ctypes.c_void_p(out_l.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(lib, None, st)
    return out_r, out_l


CASES = [
    ("tiny_k211_12", "fp64", lambda: synth.tiny_params(1, kmesh=(2, 1, 1), fft=(12,) * 3, ecut=1.6, nbands=3,
                                                        nocc=2, scale=5.0)),
    ("tiny_k112_9", "fp32", lambda: synth.tiny_params(0, kmesh=(1, 1, 2), fft=(9,) * 3, ecut=1.6, nbands=3,
                                                       nocc=2, scale=5.0)),
    ("heg_14", "fp64", lambda: synth.WORKLOADS["heg_14"]()),
]


@pytest.mark.parametrize("name,prec,make", CASES, ids=[c[0] + "_" + c[1] for c in CASES])
def test_noalloc_matches_tc_apply_on_consecutive_calls(name, prec, make):
    from paper_2302_07420_gb300.operator import Context
    p = make()
    c_phi, c_chi, occ = _inputs(p, len(name))
    d_phi = torch.from_numpy(c_phi).cuda()
    d_chi = torch.from_numpy(c_chi).cuda()
    ctx = Context(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"],
                  precision=prec)
    ref_r, ref_l = ctx.apply(d_phi, d_chi, occ)
    torch.cuda.synchronize()
    ctx.close()
    ref_r, ref_l = ref_r.cpu().numpy(), ref_l.cpu().numpy()
    scale = max(np.abs(ref_r).max(), np.abs(ref_l).max())
    lib = _lib.load()
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"],
                           precision=prec)
    for call in range(2):
        out_r, out_l = _noalloc(lib, prm, d_phi, d_chi, occ)
        torch.cuda.synchronize()
        err = max(np.abs(out_r.cpu().numpy() - ref_r).max(), np.abs(out_l.cpu().numpy() - ref_l).max()) / scale
        assert err <= TOL[prec], (name, call, err)


def test_noalloc_rejects_problems_beyond_the_static_array():
    """The 4x4x4 silicon-like workload needs far more than the array holds: refused before device work."""
    p = synth.WORKLOADS["si_k444"]()
    lib = _lib.load()
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"])
    S = make_setup(p)
    d = torch.zeros((S.Nk, S.nbands, S.npw_max), dtype=torch.complex128, device="cuda")
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    out = torch.empty_like(d)
    st = lib.tc_apply_noalloc(ctypes.byref(prm), ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                              occ.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(out.data_ptr()),
                              None, None)
    assert st == _lib.TC_ERR_UNSUPPORTED
    assert b"TC_NOALLOC_MAX_BYTES" in lib.tc_last_error(None)


def test_noalloc_larger_smaller_larger_and_one_side_keep_matching_tc_apply():
    """One process: a 16^3 FP64 case, a 9^3 FP32 case, the 16^3 case again (the shared array holds the
    smaller call's contents in between), and one call with out_L = NULL; each equals tc_apply.  Free
    device memory does not change from one call to the next: the calls allocate nothing."""
    from paper_2302_07420_gb300.operator import Context
    lib = _lib.load()
    runs = []
    for name, prec, make in (CASES[2], CASES[1]):
        p = make()
        c_phi, c_chi, occ = _inputs(p, len(name))
        d_phi, d_chi = torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda()
        ctx = Context(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"],
                      precision=prec)
        ref_r, ref_l = ctx.apply(d_phi, d_chi, occ)
        torch.cuda.synchronize()
        ctx.close()
        prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"],
                               p["C"], precision=prec)
        runs.append((name, prec, prm, d_phi, d_chi, np.ascontiguousarray(occ, dtype=np.float64),
                     ref_r.cpu().numpy(), ref_l.cpu().numpy(), torch.empty_like(d_phi), torch.empty_like(d_chi)))
    torch.cuda.synchronize()
    free = []
    for i in (0, 1, 0, 0):
        name, prec, prm, d_phi, d_chi, occ, ref_r, ref_l, out_r, out_l = runs[i]
        one_side = len(free) == 3
        st = lib.tc_apply_noalloc(ctypes.byref(prm), ctypes.c_void_p(d_phi.data_ptr()),
                                  ctypes.c_void_p(d_chi.data_ptr()),
                                  occ.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.c_void_p(out_r.data_ptr()),
                                  None if one_side else ctypes.c_void_p(out_l.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        _lib.check(lib, None, st)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        scale = max(np.abs(ref_r).max(), np.abs(ref_l).max())
        err = np.abs(out_r.cpu().numpy() - ref_r).max() / scale
        if not one_side:
            err = max(err, np.abs(out_l.cpu().numpy() - ref_l).max() / scale)
        assert err <= TOL[prec], (name, len(free), err)
    assert free[1] == free[2] == free[3], free


def test_noalloc_refuses_a_capturing_stream():
    """The per-call uploads read host memory that lives only during the call: a call on a stream that
    is capturing a graph returns TC_ERR_STATE before any work."""
    name, prec, make = CASES[1]
    p = make()
    c_phi, c_chi, occ = _inputs(p, len(name))
    d_phi, d_chi = torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda()
    out_r, out_l = torch.empty_like(d_phi), torch.empty_like(d_chi)
    occ = np.ascontiguousarray(occ, dtype=np.float64)
    lib = _lib.load()
    prm = _lib.make_params(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"],
                           precision=prec)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            st = lib.tc_apply_noalloc(ctypes.byref(prm), ctypes.c_void_p(d_phi.data_ptr()),
                                      ctypes.c_void_p(d_chi.data_ptr()),
                                      occ.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ctypes.c_void_p(out_r.data_ptr()), ctypes.c_void_p(out_l.data_ptr()),
                                      ctypes.c_void_p(s.cuda_stream))
        finally:
            g.capture_end()
    assert st == _lib.TC_ERR_STATE
    assert b"capturing" in lib.tc_last_error(None)
