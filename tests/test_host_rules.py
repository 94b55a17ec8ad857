"""Host logic of the launch decomposition (csrc/tc_setup.cpp), on the CPU: the default partner-chunk
count (pick_split: best filled last wave of CTAs on the SMs) and the autotuner's choice among measured
counts (smallest_near_best: the smallest count within 2 % of the fastest).  A probe compiled from the
library's source answers queries; the expected values restate the two rules.
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
