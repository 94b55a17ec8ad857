"""Host logic of the launch decomposition (csrc/tc_setup.cpp), on the CPU: the default partner-chunk
count (pick_split: best filled last wave of CTAs on the SMs), the autotuner's choice among measured
counts (smallest_near_best: the smallest count within 2 % of the fastest), and the grid rules that
tc_init and tc_apply_noalloc share: the Miller span of the spheres, whether the left occupied-pair
fields are exact conjugates of the right ones (odd box or span <= n/2 - 1), and the pair-density
support length min(n, 2 span + 1) that selects the pruned pair-chain transforms, and the size of the
reflection buffer of mirrored FP64 pair chains (or none).  A probe compiled from the library's source
answers queries; the expected values restate the rules.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_07420_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("rules") / "rules_probe")
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(ROOT, "tests", "host", "rules_probe.cpp"), os.path.join(CSRC, "tc_setup.cpp")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

    def ask(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True)
        assert out.returncode == 0, out.stderr
        return [int(x) for x in out.stdout.split()]
    return ask


def _split(items, partners, sms):
    best, best_eff = 1, 0.0
    for s in range(1, min(8, partners) + 1):
        ctas = items * s
        eff = ctas / (math.ceil(ctas / sms) * sms)
        if eff > best_eff + 0.01:
            best, best_eff = s, eff
    return best


def _near(t):
    b = min(t)
    return next(i + 1 for i, x in enumerate(t) if x <= 1.02 * b)


def test_pick_split(probe):
    cases = [(items, partners, sms) for items in (1, 7, 64, 128, 256, 512, 1000) for partners in (1, 3, 8, 256)
             for sms in (1, 76, 152)]
    got = probe(["split %d %d %d" % c for c in cases])
    assert got == [_split(*c) for c in cases]
    assert _split(256, 256, 152) == got[cases.index((256, 256, 152))]
    assert all(1 <= g <= min(8, c[1]) for g, c in zip(got, cases))


def test_smallest_near_best(probe):
    rng = np.random.default_rng(7)
    cases = [list(rng.uniform(100, 110, n)) for n in (1, 2, 5, 8) for _ in range(20)]
    cases += [[254.1, 216.5, 222.9, 209.0, 212.2, 214.8, 212.5],     # measured chain + 3b4 stage times (ms)
              [167.0, 168.8, 170.7, 172.3, 173.5, 175.3, 177.4],
              [10.0, 10.2, 9.9], [10.0, 9.7, 9.9]]
    got = probe(["near %d %s" % (len(t), " ".join("%.17g" % x for x in t)) for t in cases])
    assert got == [_near(t) for t in cases]
    assert got[-4] == 4 and got[-3] == 1 and got[-2] == 1 and got[-1] == 2   # 209.0 at s = 4; 216.5 is 3.6 % off


def test_miller_span_of_oracle_spheres(probe):
    """The span of the oracle's own spheres (si_k444 cell: 8, the 24^3 support edge 17) and of
    Gamma-only HEG spheres (|n|^2 <= 16: span 8)."""
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from conftest import make_setup
    from paper_2302_07420_gb300 import synth
    lines, want = [], []
    for p in (synth.si_params(kmesh=(1, 1, 2)), synth.WORKLOADS["heg_14"](),
              synth.tiny_params(11, kmesh=(1, 1, 2), fft=(24,) * 3, ecut=6.0, nbands=3, nocc=2, scale=5.0)):
        S = make_setup(p)
        allm = np.concatenate(S.miller)
        lines.append("span %d %s" % (len(allm), " ".join("%d %d %d" % tuple(m) for m in allm)))
        want.append(int((allm.max(0) - allm.min(0)).max()))
    assert probe(lines) == want
    assert want[0] == 8 and want[1] == 8


def test_grid_rules(probe):
    cases = [(n, s) for n in (9, 12, 15, 16, 24, 25, 48) for s in range(0, 26)]
    out = probe(["grid %d %d" % c for c in cases])
    pairs = list(zip(out[0::2], out[1::2]))
    for (n, s), (clear, sup) in zip(cases, pairs):
        assert clear == int(n % 2 == 1 or s <= n // 2 - 1), (n, s)
        assert sup == min(n, 2 * s + 1), (n, s)
    # the si_k444 grid: span 8 on 24^3 is clear of the Nyquist planes and fills the 17-index support
    assert pairs[cases.index((24, 8))] == (1, 17)
    assert pairs[cases.index((24, 9))] == (1, 19) and pairs[cases.index((24, 12))] == (0, 24)


def test_mirror_buffer_rule(probe):
    """FP64 mesh contexts on the pruned transforms: (Nk no)^2 x 2 x L^3 x 16 bytes when at most a quarter
    of the free memory; nothing in FP32, with band points, without pruned transforms or when it does not fit."""
    gib = 1 << 30
    cases = [(1, 0, 17, 17, 64, 4, 280 * gib), (0, 0, 17, 17, 64, 4, 280 * gib), (1, 1, 17, 17, 64, 4, 280 * gib),
             (1, 0, 0, 21, 64, 4, 280 * gib), (1, 0, 17, 19, 64, 4, 280 * gib), (1, 0, 17, 17, 64, 4, 30 * gib),
             (1, 0, 13, 13, 2, 2, 1 * gib), (1, 0, 17, 9, 2, 3, 4 * gib)]
    got = probe(["mirror %d %d %d %d %d %d %d" % c for c in cases])

    def rule(fp64, nkb, L, sup, nk, no, free):
        if not fp64 or nkb > 0 or L <= 0 or sup > L:
            return 0
        b = (nk * no) ** 2 * 2 * L ** 3 * 16
        return b if b <= free // 4 else 0
    assert got == [rule(*c) for c in cases]
    assert got[0] == 256 ** 2 * 2 * 17 ** 3 * 16    # si_k444 FP64: 10.3 GB
    assert got[5] == 0                              # 30 GiB free: does not fit in a quarter
