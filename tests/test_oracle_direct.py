"""Brute force: the FFT route equals direct cyclic sums in reciprocal space (pin P10).

``DirectBackend`` holds every field by its Fourier coefficients and forms each
pointwise product as a cyclic convolution summed term by term; no FFT is used.
"""
import numpy as np
import pytest

from conftest import make_setup
from oracle import operator as OP
from oracle.backends import DirectBackend
from paper_2302_07420_gb300 import synth


@pytest.mark.parametrize("seed,kmesh,fft", [(0, (1, 1, 2), (6, 5, 6)), (1, (2, 1, 1), (5, 6, 5))])
@pytest.mark.parametrize("left", [False, True])
def test_fft_route_equals_direct_sums(seed, kmesh, fft, left):
    p = synth.tiny_params(seed, kmesh=kmesh, fft=fft, ecut=1.5, nbands=3, nocc=2, scale=5.0)
    S = make_setup(p)
    assert max(np.abs(m).max() for m in S.miller) >= 1
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + 50 + seed, [S.kpG(k) for k in range(S.Nk)],
                                         S.npw_max, S.nbands, perturb=0.2)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    occ[:, 1] = 0.7
    a = OP.apply_operator(S, c_phi, c_chi, occ, left=left)
    b = OP.apply_operator(S, c_phi, c_chi, occ, left=left, backend=DirectBackend)
    scale = max(np.abs(OP.total(a)).max(), 1e-8)
    for t in OP.TERMS:
        assert np.abs(a[t]).max() > 1e-8 * scale or t in (), t
        np.testing.assert_allclose(a[t], b[t], rtol=0, atol=1e-12 * scale, err_msg=t)
