"""tc_energy_grad and the autograd Function on the GPU.

* parity with the FP64 oracle gradient (oracle/gradient.py) on small cells and
  against stored oracle values for the silicon-like cell on a 2x2x2 mesh;
* the full-size silicon-like workload (4x4x4 mesh, 24^3 box, FP64) against
  central differences of the GPU energy (step 1e-4) to a relative 1e-6;
* torch.autograd.gradcheck of the autograd Function;
* the context's tables are restored after the parameter passes.
"""
import ctypes
import json
import os

import numpy as np
import pytest

from conftest import make_setup
from oracle import gradient as GR
from paper_2302_07420_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))

TOL_ORB64 = 1e-11     # relative to the largest gradient coefficient, as the operator parity
TOL_PAR64 = 1e-9      # dE/dA, dE/dC: difference of two FP64 energies


def _ctx(p, **kw):
    from paper_2302_07420_gb300.operator import Context
    args = dict(lattice=p["lattice"], kmesh=p["kmesh"], ecut=p["ecut"], fft=p["fft"], nbands=p["nbands"],
                nocc=p["nocc"], A=p["A"], C=p["C"])
    args.update(kw)
    return Context(**args)


def tiny_case(seed, kmesh, fft, fill=(1.0, 0.6), **kw):
    p = synth.tiny_params(seed, kmesh=kmesh, fft=(fft,) * 3, ecut=1.6, nbands=3, nocc=2, scale=5.0)
    S = make_setup(p, **kw)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 400 + seed, [S.kpG(k) for k in range(S.Nk)], S.npw_max,
                                         S.nbands, perturb=0.1)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, :2] = np.asarray(fill)[None]
    return p, S, c_phi, c_chi, occ


CASES = [(0, (1, 1, 2), 9, 1, 1.0), (1, (2, 1, 1), 12, 1, 2.0), (2, (1, 2, 1), 15, 0, 1.0)]


@pytest.mark.parametrize("seed,kmesh,fft,div,uf", CASES)
def test_energy_grad_matches_oracle_fp64(seed, kmesh, fft, div, uf):
    p, S, c_phi, c_chi, occ = tiny_case(seed, kmesh, fft, div_correction=div, ushort_factor=uf)
    ref_phi, ref_chi = GR.orbital_gradient(S, c_phi, c_chi, occ)
    ref_par = GR.param_gradient(S, c_phi, c_chi, occ)
    ctx = _ctx(p, div_correction=div, ushort_factor=uf)
    g_phi, g_chi, dA, dC = ctx.energy_grad(torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda(), occ)
    ctx.close()
    scale = max(np.abs(ref_phi).max(), np.abs(ref_chi).max())
    assert np.abs(g_phi.cpu().numpy() - ref_phi).max() / scale < TOL_ORB64
    assert np.abs(g_chi.cpu().numpy() - ref_chi).max() / scale < TOL_ORB64
    for name, got in (("A", dA), ("C", dC)):
        ref = np.array(ref_par[name])
        assert np.all(np.abs(got - ref) <= TOL_PAR64 * np.maximum(np.abs(ref), 1e-2)), (name, got, ref)


def test_energy_grad_fp32_path():
    """FP32 FFTs and pair products: orbital gradient within the operator bound, parameters within 1e-4."""
    p, S, c_phi, c_chi, occ = tiny_case(1, (2, 1, 1), 12)
    ref_phi, ref_chi = GR.orbital_gradient(S, c_phi, c_chi, occ)
    ref_par = GR.param_gradient(S, c_phi, c_chi, occ)
    ctx = _ctx(p, precision="fp32")
    g_phi, g_chi, dA, dC = ctx.energy_grad(torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda(), occ)
    ctx.close()
    scale = max(np.abs(ref_phi).max(), np.abs(ref_chi).max())
    assert np.abs(g_phi.cpu().numpy() - ref_phi).max() / scale < 1e-5
    assert np.abs(g_chi.cpu().numpy() - ref_chi).max() / scale < 1e-5
    for name, got in (("A", dA), ("C", dC)):
        ref = np.array(ref_par[name])
        assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(np.abs(ref), 1e-1)), (name, got, ref)


def test_host_pointers_and_tables_restored():
    """Host outputs equal device outputs, and tc_apply after tc_energy_grad is bit-identical to before."""
    p, S, c_phi, c_chi, occ = tiny_case(0, (1, 1, 2), 9)
    ctx = _ctx(p)
    d_phi, d_chi = torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda()
    r0, l0 = ctx.apply(d_phi, d_chi, occ)
    r0, l0 = r0.cpu().numpy(), l0.cpu().numpy()
    g_phi, g_chi, dA, dC = ctx.energy_grad(d_phi, d_chi, occ)
    h_phi, h_chi = np.empty_like(c_phi), np.empty_like(c_chi)
    occ_c = np.ascontiguousarray(occ)
    dA2, dC2 = (ctypes.c_double * 2)(), (ctypes.c_double * 2)()
    st = ctx.lib.tc_energy_grad(ctx.h, ctypes.c_void_p(c_phi.ctypes.data), ctypes.c_void_p(c_chi.ctypes.data),
                                occ_c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.c_void_p(h_phi.ctypes.data), ctypes.c_void_p(h_chi.ctypes.data), dA2, dC2, None)
    assert st == _lib.TC_OK
    assert np.array_equal(h_phi, g_phi.cpu().numpy()) and np.array_equal(h_chi, g_chi.cpu().numpy())
    assert list(dA2) == list(dA) and list(dC2) == list(dC)
    r1, l1 = ctx.apply(d_phi, d_chi, occ)
    assert np.array_equal(r1.cpu().numpy(), r0) and np.array_equal(l1.cpu().numpy(), l0)
    ctx.close()


def test_argument_errors():
    p, S, c_phi, c_chi, occ = tiny_case(0, (1, 1, 2), 9)
    d_phi, d_chi = torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda()
    ctx = _ctx(p)
    bad = occ.copy()
    bad[:, 2] = 0.5
    with pytest.raises(_lib.TCError) as e:
        ctx.energy_grad(d_phi, d_chi, bad)
    assert e.value.status == _lib.TC_ERR_ARG
    ctx.close()
    ctx = _ctx(p, term_mask=1 << 3)
    with pytest.raises(_lib.TCError) as e:
        ctx.energy_grad(d_phi, d_chi, occ, params=False)
    assert e.value.status == _lib.TC_ERR_UNSUPPORTED
    _, _, dA, dC = ctx.energy_grad(d_phi, d_chi, occ, orbitals=False)   # parameters only: any term subset
    assert np.all(np.isfinite(dA)) and np.all(np.isfinite(dC))
    ctx.close()


def test_si_k222_against_oracle_values():
    """Silicon-like cell, 2x2x2 mesh, 24^3 box, FP64: gradient vs tests/golden/si_k222_grad.json (oracle)."""
    g = json.load(open(os.path.join(HERE, "golden", "si_k222_grad.json")))
    p = synth.si_params(kmesh=(2, 2, 2))
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(g["seed"], [S.kpG(k) for k in range(S.Nk)], S.npw_max, S.nbands)
    probe = np.array([c_phi[k, b, i] for k, b, i in g["input_probe"]["index"]])
    assert np.abs(probe - np.array(g["input_probe"]["phi"]).view(complex).ravel()).max() < 1e-13
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    ctx = _ctx(p)
    d_phi, d_chi = torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda()
    g_phi, g_chi, dA, dC = ctx.energy_grad(d_phi, d_chi, occ)
    E = ctx.energy(d_phi, d_chi, occ)
    ctx.close()
    assert abs(E - g["energy"]) < 1e-11 * abs(g["energy"])
    gp, gc = g_phi.cpu().numpy(), g_chi.cpu().numpy()
    refs = {k: (np.array(g["g_phi"][str(k)]).view(complex).reshape(S.nbands, -1),
                np.array(g["g_chi"][str(k)]).view(complex).reshape(S.nbands, -1)) for k in g["sample_k"]}
    scale = max(max(np.abs(a).max(), np.abs(b).max()) for a, b in refs.values())
    for k, (rp, rc) in refs.items():
        assert np.abs(gp[k] - rp).max() / scale < TOL_ORB64
        assert np.abs(gc[k] - rc).max() / scale < TOL_ORB64
    for name, got in (("dE_dA", dA), ("dE_dC", dC)):
        ref = np.array(g[name])
        assert np.all(np.abs(got - ref) <= TOL_PAR64 * np.abs(ref)), (name, got, ref)


def test_full_size_gradient_against_central_differences():
    """4x4x4 mesh, 24^3 box, FP64: dE/dA, dE/dC and two orbital directions per set vs differences (h = 1e-4)."""
    p = synth.WORKLOADS["si_k444"]()
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 1, [S.kpG(k) for k in range(S.Nk)], S.npw_max, S.nbands)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    d_phi, d_chi = torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda()
    ctx = _ctx(p)
    g_phi, g_chi, dA, dC = ctx.energy_grad(d_phi, d_chi, occ)
    h = 1e-4
    rng = np.random.default_rng(3)
    mask = np.zeros((S.Nk, 1, S.npw_max))
    for k in range(S.Nk):
        mask[k, :, : S.npw[k]] = 1.0
    for which, grad in (("phi", g_phi), ("chi", g_chi)):
        for _ in range(2):
            d = (rng.standard_normal(c_phi.shape) + 1j * rng.standard_normal(c_phi.shape)) * mask
            d /= np.linalg.norm(d)
            dd = torch.from_numpy(d).cuda()
            if which == "phi":
                Ep, Em = ctx.energy(d_phi + h * dd, d_chi, occ), ctx.energy(d_phi - h * dd, d_chi, occ)
            else:
                Ep, Em = ctx.energy(d_phi, d_chi + h * dd, occ), ctx.energy(d_phi, d_chi - h * dd, occ)
            fd = (Ep - Em) / (2 * h)
            val = float(torch.real(torch.sum(torch.conj(grad) * dd)))
            assert abs(val - fd) < 1e-6 * abs(fd), (which, val, fd)
    ctx.close()
    for name, got in (("A", dA), ("C", dC)):
        for s in range(2):
            vals = []
            for sg in (1, -1):
                A, C = list(p["A"]), list(p["C"])
                (A if name == "A" else C)[s] += sg * h
                c2 = _ctx(p, A=A, C=C)
                vals.append(c2.energy(d_phi, d_chi, occ))
                c2.close()
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(got[s] - fd) < 1e-6 * abs(fd), (name, s, got[s], fd)


def test_autograd_function_gradcheck():
    from paper_2302_07420_gb300.autograd import TCEnergyModel
    p, S, c_phi, c_chi, occ = tiny_case(0, (1, 1, 2), 9, fill=(1.0, 0.7))
    model = TCEnergyModel(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"])
    phi = torch.from_numpy(c_phi).cuda().requires_grad_()
    chi = torch.from_numpy(c_chi).cuda().requires_grad_()
    A = torch.tensor(p["A"], dtype=torch.float64, requires_grad=True)
    C = torch.tensor(p["C"], dtype=torch.float64, requires_grad=True)
    f = lambda a, b, x, y: model.energy(a, b, x, y, occ)
    assert torch.autograd.gradcheck(f, (phi, chi, A, C), eps=1e-6, atol=1e-7, rtol=1e-5)
    E = f(phi, chi, A, C)
    E.backward()
    ctx = _ctx(p)
    g_phi, g_chi, dA, dC = ctx.energy_grad(phi.detach(), chi.detach(), occ)
    ctx.close()
    model.close()
    assert torch.equal(phi.grad, g_phi) and torch.equal(chi.grad, g_chi)
    assert np.array_equal(A.grad.numpy(), dA) and np.array_equal(C.grad.numpy(), dC)
