"""The bench's unit of work, on the CPU (no GPU needed).

One step applies the operator to every right and left orbital of the 4x4x4 silicon-like cell
(64 k-points, 4 bands, 4 occupied): each output orbital j pairs with every occupied partner q in the
pair chains, (64 * 4) * (64 * 4) pairs per side, and each ordered pair of occupied orbitals enters the
occupied-pair stage, (64 * 4)^2 per side; both sides together are 262,144 pair convolutions.  The
roofline's algorithmic work per pair chain is 14 complex transforms of 5 N log2 N flops on the 24^3 box.
"""
import math

import bench


def test_pairs_per_step_of_the_bench_workload():
    assert bench.pairs_per_apply(64, 4, 4) == 262144
    assert bench.pairs_per_apply(1, 7, 7) == 2 * (49 + 49)          # the Gamma-only HEG of 14 electrons
    assert bench.pairs_per_apply(8, 6, 4) == 2 * (48 * 32 + 32 * 32)


def test_pair_chain_flop_convention():
    N = 24 ** 3
    per_chain = bench.FFTS_PER_PAIR_CHAIN * 5.0 * N * math.log2(N)
    assert bench.FFTS_PER_PAIR_CHAIN == 14
    assert abs(per_chain - 13.31e6) < 0.01e6          # 14 x 0.951 MFLOP
    # one launch of the 4x4x4 workload covers both sides' 131,072 chains: 1.7446 TFLOP
    assert abs(2 * 256 * 256 * per_chain - 1.7446e12) < 0.001e12
