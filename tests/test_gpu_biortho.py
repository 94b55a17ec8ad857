"""tc_biorthonormalize against oracle/biortho.py (FP64) through the C ABI."""
import numpy as np
import pytest

from conftest import make_setup
from oracle import biortho as BO
from paper_2302_07420_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _raw(S, seed):
    rng = np.random.default_rng(seed)
    shape = (S.Nk, S.nbands, S.npw_max)
    phi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    chi = phi + 0.3 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    for k in range(S.Nk):
        phi[k, :, S.npw[k]:] = 0.0
        chi[k, :, S.npw[k]:] = 0.0
    return phi, chi


def _ctx(p):
    from paper_2302_07420_gb300.operator import Context
    return Context(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"])


@pytest.mark.parametrize("name", ["tiny", "si_k222"])
def test_matches_oracle_device_and_host(name):
    p = (synth.tiny_params(2, kmesh=(1, 2, 2), fft=(12,) * 3, ecut=1.6, nbands=5, nocc=3, scale=5.0)
         if name == "tiny" else synth.si_params(kmesh=(2, 2, 2)))
    S = make_setup(p)
    phi0, chi0 = _raw(S, 17)
    ref_phi, ref_chi = BO.biorthonormalize(phi0, chi0)
    ctx = _ctx(p)
    dphi, dchi = torch.from_numpy(phi0).cuda(), torch.from_numpy(chi0).cuda()
    ctx.biorthonormalize(dphi, dchi)
    hphi, hchi = phi0.copy(), chi0.copy()
    ctx.biorthonormalize(hphi, hchi)
    ctx.close()
    for got_phi, got_chi in ((dphi.cpu().numpy(), dchi.cpu().numpy()), (hphi, hchi)):
        assert np.abs(got_phi - ref_phi).max() < 1e-12 * np.abs(ref_phi).max()
        assert np.abs(got_chi - ref_chi).max() < 1e-11 * np.abs(ref_chi).max()
        for k in range(S.Nk):
            np.testing.assert_allclose(np.conj(got_chi[k]) @ got_phi[k].T, np.eye(S.nbands), atol=1e-12)


def test_singular_overlap_is_reported():
    p = synth.tiny_params(2, kmesh=(1, 1, 2), fft=(9,) * 3, ecut=1.6, nbands=3, nocc=2, scale=5.0)
    S = make_setup(p)
    phi0, chi0 = _raw(S, 3)
    chi0[1, 2] = chi0[1, 0]        # two equal left orbitals at k = 1: M is singular there
    ctx = _ctx(p)
    with pytest.raises(_lib.TCError) as e:
        ctx.biorthonormalize(torch.from_numpy(phi0).cuda(), torch.from_numpy(chi0).cuda())
    assert e.value.status == _lib.TC_ERR_ARG and "k-point 1" in str(e.value)
    ctx.close()
