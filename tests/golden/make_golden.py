"""Writes oracle expected values for the full-size workloads (calls only oracle/).

si_k444: silicon-like FCC cell, a = 10.26 bohr, 4x4x4 mesh, ecut 7.5 Ha, box 24^3,
4 occupied bands, inputs from paper_2302_07420_gb300.synth (seed 230207420 + 1).
Stored: out_R / out_L (every term summed) at the sampled k-points, E_TC and its
per-term split, and a few input coefficients to confirm that the regenerated
inputs are the ones used here.

si_k222_grad: the same cell, box and recipe on a 2x2x2 mesh (seed 230207420 + 5):
the energy gradient of oracle/gradient.py -- g_phi, g_chi at the sampled
k-points and dE/dA, dE/dC -- and E_TC.

si_k444_band: the si_k444 partners (same seed) and one band-structure k-point
off the mesh, k_b = (0.13, 0.27, -0.31) in the reciprocal basis, carrying 4
seeded random biorthonormal band orbitals on its own sphere (seed 230207420 + 6,
all occupied, f = 1): out_R / out_L of oracle/band.py at k_b (every term and
band correction summed), Gamma_b and W.

Run:  python tests/golden/make_golden.py si_k444
      python tests/golden/make_golden.py si_k222_grad
      python tests/golden/make_golden.py si_k444_band
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import band as BD  # noqa: E402
from oracle import gradient as GR  # noqa: E402
from oracle import operator as OP  # noqa: E402
from oracle.cell import Setup  # noqa: E402
from paper_2302_07420_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SAMPLE_K = {"si_k444": [0, 21, 42], "si_k222_grad": [0, 5]}
SEED_OFFSET = {"si_k444": 1, "si_k222_grad": 5, "si_k444_band": 6}
K_BAND = [0.13, 0.27, -0.31]


def inputs(name):
    p = synth.WORKLOADS[name]() if name in synth.WORKLOADS else synth.si_params(kmesh=(2, 2, 2))
    S = Setup(p["lattice"], p["kmesh"], p["ecut"], p["fft"], p["nbands"], p["nocc"], p["A"], p["C"])
    c_phi, c_chi = synth.random_orbitals(synth.SEED0 + SEED_OFFSET[name], [S.kpG(k) for k in range(S.Nk)],
                                         S.npw_max, S.nbands)
    occ = synth.occupations(S.Nk, S.nbands, S.nocc)
    return p, S, c_phi, c_chi, occ


def cplx_list(a):
    return [[float(x.real), float(x.imag)] for x in np.asarray(a).ravel()]


def main_grad(name):
    t0 = time.time()
    p, S, c_phi, c_chi, occ = inputs(name)
    ks = SAMPLE_K[name]
    g_phi, g_chi = GR.orbital_gradient(S, c_phi, c_chi, occ)
    pg = GR.param_gradient(S, c_phi, c_chi, occ)
    E = OP.energy_terms(S, c_phi, c_chi, occ)["total"]
    doc = {
        "workload": name,
        "source": "oracle/ (tests/golden/make_golden.py)",
        "seed": synth.SEED0 + SEED_OFFSET[name],
        "shape": [S.Nk, S.nbands, S.npw_max],
        "sample_k": ks,
        "input_probe": {"index": [[k, b, 5] for k in ks for b in range(S.nbands)],
                        "phi": cplx_list([c_phi[k, b, 5] for k in ks for b in range(S.nbands)])},
        "g_phi": {str(k): cplx_list(g_phi[k]) for k in ks},
        "g_chi": {str(k): cplx_list(g_chi[k]) for k in ks},
        "dE_dA": pg["A"],
        "dE_dC": pg["C"],
        "energy": E,
        "oracle_seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(doc, f)
    print("wrote", name, "in %.0f s" % (time.time() - t0))


def band_inputs():
    p, S, c_phi, c_chi, occ = inputs("si_k444")
    SB = BD.BandSetup(S, K_BAND)
    kb = S.Nk
    b_phi, b_chi = synth.random_orbitals(synth.SEED0 + SEED_OFFSET["si_k444_band"], [SB.kpG(kb)], SB.npw_max,
                                         S.nbands)
    b_occ = synth.occupations(1, S.nbands, S.nocc)
    return p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ


def main_band(name):
    t0 = time.time()
    p, S, SB, c_phi, c_chi, occ, b_phi, b_chi, b_occ = band_inputs()
    r = OP.total(BD.band_apply(S, c_phi, c_chi, occ, K_BAND, b_phi, b_chi, b_occ, left=False))
    l = OP.total(BD.band_apply(S, c_phi, c_chi, occ, K_BAND, b_phi, b_chi, b_occ, left=True))
    npw = int(SB.npw[S.Nk])
    doc = {
        "workload": name,
        "source": "oracle/ (tests/golden/make_golden.py)",
        "seed_partners": synth.SEED0 + SEED_OFFSET["si_k444"],
        "seed_band": synth.SEED0 + SEED_OFFSET[name],
        "k_band_frac": K_BAND,
        "npw_band": npw,
        "miller_band": SB.miller[S.Nk].tolist(),
        "input_probe": {"index": [[b, 5] for b in range(S.nbands)],
                        "phi": cplx_list([b_phi[0, b, 5] for b in range(S.nbands)]),
                        "chi": cplx_list([b_chi[0, b, 5] for b in range(S.nbands)])},
        "gamma_b": SB.gamma_b[0],
        "W": [float(x) for x in SB.W[0]],
        "out_R": cplx_list(r[0][:, :npw]),
        "out_L": cplx_list(l[0][:, :npw]),
        "oracle_seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(doc, f)
    print("wrote", name, "in %.0f s" % (time.time() - t0))


def main(name):
    if name.endswith("_grad"):
        return main_grad(name)
    if name.endswith("_band"):
        return main_band(name)
    t0 = time.time()
    p, S, c_phi, c_chi, occ = inputs(name)
    ks = SAMPLE_K[name]
    right = OP.apply_operator(S, c_phi, c_chi, occ, left=False)            # all k: needed for E
    E = OP.energy_terms(S, c_phi, c_chi, occ, res=right)
    left = OP.apply_operator(S, c_phi, c_chi, occ, left=True, kpoints=ks)
    out_r, out_l = OP.total(right), OP.total(left)
    doc = {
        "workload": name,
        "source": "oracle/ (tests/golden/make_golden.py)",
        "seed": synth.SEED0 + SEED_OFFSET[name],
        "shape": [S.Nk, S.nbands, S.npw_max],
        "sample_k": ks,
        "input_probe": {"index": [[k, b, 5] for k in ks for b in range(S.nbands)],
                        "phi": cplx_list([c_phi[k, b, 5] for k in ks for b in range(S.nbands)]),
                        "chi": cplx_list([c_chi[k, b, 5] for k in ks for b in range(S.nbands)])},
        "out_R": {str(k): cplx_list(out_r[k]) for k in ks},
        "out_L": {str(k): cplx_list(out_l[k]) for k in ks},
        "energy": E,
        "oracle_seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(doc, f)
    print("wrote", name, "in %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "si_k444")
