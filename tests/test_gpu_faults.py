"""Host-side fault injection (TC_FAULT) on the GPU.

The injected failures happen in the C wrappers before any device work: the
calls return their status, the outputs stay untouched and the context stays
usable.  No device fault, trap or hang is involved.
"""
import numpy as np
import pytest

from conftest import make_setup
from paper_2302_07420_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(p, **kw):
    from paper_2302_07420_gb300.operator import Context
    args = dict(lattice=p["lattice"], kmesh=p["kmesh"], ecut=p["ecut"], fft=p["fft"], nbands=p["nbands"],
                nocc=p["nocc"], A=p["A"], C=p["C"])
    args.update(kw)
    return Context(**args)


def test_injected_faults_leave_outputs_and_context_intact(monkeypatch):
    from paper_2302_07420_gb300 import _lib
    p = synth.tiny_params(8, kmesh=(1, 1, 2), fft=(12,) * 3, ecut=1.6, nbands=3, nocc=2, scale=5.0)
    S = make_setup(p)
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 400, [S.kpG(k) for k in range(S.Nk)], S.npw_max, S.nbands,
                                         perturb=0.1)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    ctx = _ctx(p)
    try:
        a, b = torch.from_numpy(c_phi).cuda(), torch.from_numpy(c_chi).cuda()
        r0, l0 = ctx.apply(a, b, occ)
        r0, l0 = r0.clone(), l0.clone()
        e0 = ctx.energy(a, b, occ)
        out_r, out_l = torch.full_like(a, 7.0), torch.full_like(a, 7.0)
        for kind, status in (("launch", _lib.TC_ERR_CUDA), ("timeout", _lib.TC_ERR_TIMEOUT)):
            monkeypatch.setenv("TC_FAULT", kind)
            with pytest.raises(_lib.TCError) as e:
                ctx.apply(a, b, occ, out_r, out_l)
            assert e.value.status == status and "TC_FAULT" in str(e.value)
            with pytest.raises(_lib.TCError) as e:
                ctx.energy(a, b, occ)
            assert e.value.status == status
            with pytest.raises(_lib.TCError) as e:
                ctx.davidson_step(a, b, occ)
            assert e.value.status == status
            torch.cuda.synchronize()
            assert bool((out_r == 7.0).all()) and bool((out_l == 7.0).all())
        monkeypatch.setenv("TC_FAULT", "alloc")
        with pytest.raises(_lib.TCError) as e:
            _ctx(p)
        assert e.value.status == _lib.TC_ERR_OOM
        monkeypatch.delenv("TC_FAULT")
        r1, l1 = ctx.apply(a, b, occ, out_r, out_l)
        torch.cuda.synchronize()
        assert torch.equal(r1, r0) and torch.equal(l1, l0)
        assert ctx.energy(a, b, occ) == e0
    finally:
        ctx.close()
