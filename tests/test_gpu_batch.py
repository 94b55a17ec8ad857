"""Batched cells (tc_init_batch / tc_apply_batch) on the GPU.

Cells from the HEG batch recipe (synth.heg_batch: uneven boxes 16^3-32^3,
1-8 k-points, 7-33 plane waves per k), FP32:
* every cell's output equals a single-cell tc_apply of the same inputs bit for bit (single-cell
  contexts without the mirrored pair chains, TC_FAULT=nomirror, as batch cells run them);
* plane-wave orbitals: every output is diagonal in momentum and out_L = out_R (BITC = TC);
* the two cheapest cells against the FP64 oracle (1e-5), and for every box size of the recipe the
  cheapest cell of the 256, batched together, against the oracle (1e-5);
* a second call replays the captured graph with identical results;
* error paths of the batch API.
"""
import ctypes

import numpy as np
import pytest

from conftest import make_setup
from oracle import operator as OP
from paper_2302_07420_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NCELL = 12


def _inputs(cells):
    out = []
    for p in cells:
        S = make_setup(p)
        c = synth.heg_kpoint_orbitals([S.kpG(k) for k in range(S.Nk)], S.miller, S.npw_max, S.nocc)
        occ = synth.occupations(S.Nk, S.nbands, S.nocc)
        out.append((S, c, occ))
    return out


@pytest.fixture(scope="module")
def batch():
    from paper_2302_07420_gb300.operator import BatchContext
    cells = synth.heg_batch(256)[:NCELL]
    data = _inputs(cells)
    bc = BatchContext(cells, precision="fp32")
    for i, (S, c, occ) in enumerate(data):
        nk, npw_max, npw, miller = bc.layouts[i]
        assert nk == S.Nk and npw_max == S.npw_max and npw.tolist() == S.npw.tolist()
    d = [torch.from_numpy(c).cuda() for _, c, _ in data]
    out_r, out_l = bc.apply(d, d, [o for _, _, o in data])
    torch.cuda.synchronize()
    res = [(r.cpu().numpy(), l.cpu().numpy()) for r, l in zip(out_r, out_l)]
    yield cells, data, bc, d, res
    bc.close()


def test_batch_equals_single_cell_calls(batch, monkeypatch):
    from paper_2302_07420_gb300.operator import Context
    cells, data, bc, d, res = batch
    monkeypatch.setenv("TC_FAULT", "nomirror")   # batch cells hold no reflection buffer
    for i, (p, (S, c, occ)) in enumerate(zip(cells, data)):
        ctx = Context(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"],
                      precision="fp32")
        r, l = ctx.apply(d[i], d[i], occ)
        torch.cuda.synchronize()
        ctx.close()
        assert np.array_equal(r.cpu().numpy(), res[i][0]), i
        assert np.array_equal(l.cpu().numpy(), res[i][1]), i


def test_plane_waves_stay_diagonal_and_bitc_equals_tc(batch):
    cells, data, bc, d, res = batch
    for i, (S, c, occ) in enumerate(data):
        r, l = res[i]
        mask = np.abs(c) > 0
        diag = np.abs(r[mask]).max()
        assert np.abs(np.where(mask, 0, r)).max() < 1e-5 * diag, i
        assert np.abs(l - r).max() < 1e-5 * diag, i


def test_cheapest_cells_against_the_oracle(batch):
    cells, data, bc, d, res = batch
    cost = [S.Nk ** 2 * S.nocc ** 2 * S.N for S, _, _ in data]
    for i in np.argsort(cost)[:2]:
        S, c, occ = data[i]
        ref_r, ref_l = OP.tc_apply(S, c, c, occ)
        scale = np.abs(ref_r).max()
        assert np.abs(res[i][0] - ref_r).max() / scale < 1e-5, i
        assert np.abs(res[i][1] - ref_l).max() / scale < 1e-5, i


def test_replay_and_tuning_info(batch):
    cells, data, bc, d, res = batch
    out_r, out_l = bc.apply(d, d, [o for _, _, o in data])
    torch.cuda.synchronize()
    for i in range(NCELL):
        assert np.array_equal(out_r[i].cpu().numpy(), res[i][0])
    ncell, lanes, lanes_max, tune = bc.info()
    assert ncell == NCELL and lanes in tune and 1 in tune and lanes <= lanes_max
    assert tune[lanes] == min(tune.values())


def test_batch_error_paths(batch):
    from paper_2302_07420_gb300.operator import BatchContext
    cells, data, bc, d, res = batch
    lib = bc.lib
    cell = ctypes.c_void_p()
    assert lib.tc_batch_cell(bc.h, 0, ctypes.byref(cell)) == _lib.TC_OK
    assert lib.tc_destroy(cell) == _lib.TC_ERR_STATE               # owned by the batch
    assert lib.tc_batch_cell(bc.h, NCELL, ctypes.byref(cell)) == _lib.TC_ERR_ARG
    occ = np.ones(8)
    st = lib.tc_apply(bc.h, None, None, occ.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, None, None)
    assert st == _lib.TC_ERR_STATE                                  # single-cell call on a batch
    mixed = [dict(cells[0]), dict(cells[1])]
    prm = (_lib.tc_params * 2)(*[_lib.make_params(*[c[k] for k in ("lattice", "kmesh", "ecut", "fft", "nbands",
                                                                       "nocc", "A", "C")], precision=pr)
                                 for c, pr in zip(mixed, ("fp32", "fp64"))])
    h = ctypes.c_void_p()
    assert lib.tc_init_batch(2, prm, ctypes.byref(h)) == _lib.TC_ERR_ARG
    with pytest.raises(_lib.TCError):
        bc.apply([torch.from_numpy(c) for _, c, _ in data], d, [o for _, _, o in data])   # host arrays


def test_one_cell_of_every_box_size_against_the_oracle():
    """For each box size of the 256-cell recipe (16^3 .. 32^3: shared-memory, pruned-free and
    global-scratch kernels) the cheapest cell, the eight batched in one graph, against the oracle."""
    from paper_2302_07420_gb300.operator import BatchContext
    allc = synth.heg_batch(256)
    best = {}
    for i, p in enumerate(allc):
        n = p["fft"][0]
        cost = int(np.prod(p["kmesh"])) ** 2 * p["nocc"] ** 2 * n ** 3
        if n not in best or cost < best[n][1]:
            best[n] = (i, cost)
    sizes = sorted(best)
    assert sizes == [16, 18, 20, 24, 25, 27, 30, 32]
    cells = [allc[best[n][0]] for n in sizes]
    data = _inputs(cells)
    bc = BatchContext(cells, precision="fp32")
    try:
        d = [torch.from_numpy(c).cuda() for _, c, _ in data]
        out_r, out_l = bc.apply(d, d, [o for _, _, o in data])
        torch.cuda.synchronize()
        res = [(r.cpu().numpy(), l.cpu().numpy()) for r, l in zip(out_r, out_l)]
    finally:
        bc.close()
    for n, (S, c, occ), (r, l) in zip(sizes, data, res):
        ref_r, ref_l = OP.tc_apply(S, c, c, occ)
        scale = np.abs(ref_r).max()
        assert np.abs(r - ref_r).max() / scale < 1e-5, n
        assert np.abs(l - ref_l).max() / scale < 1e-5, n
