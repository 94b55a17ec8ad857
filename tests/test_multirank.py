"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1).

The work shards into independent replicas (no collective on the data path),
so the only multi-rank steps are the barrier, the max-over-ranks time and the
whole-job value, and the reference arm running on rank 0 alone.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(1.0 + rank, dist)              # rank r took 1 + r seconds
        v = bench.job_value(world, 1000, 10, t)
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r\n" % (t, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    got = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(world)]
    for t, v in got:
        assert float(t) == 2.0                                  # the slowest rank's time, on every rank
        assert float(v) == 2 * 1000 * 10 / 2.0                  # units of all ranks / that time


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_value(1, 262144, 10, 4.0) == 262144 * 10 / 4.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_value_is_pairs_over_seconds(monkeypatch, capsys):
    """The reference line's value is the pairs of all timed steps over their total seconds."""
    import argparse
    import json
    sys.path.insert(0, ROOT)
    import bench
    secs = iter([9.0, 2.0, 3.0])                 # one warm-up, two timed steps

    def fake(nsteps=3, kmesh=(2, 1, 1), workers=None):
        s = next(secs)
        return 256 / s, {"cores": 4, "sample": "fake", "seconds": s}
    monkeypatch.setattr(bench, "oracle_sample_pairs_per_s", fake)
    monkeypatch.delenv("RANK", raising=False)
    bench.run_reference(argparse.Namespace(warmup=1, steps=2, gpus=1))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert abs(line["value"] - 2 * 256 / 5.0) < 1e-9
    assert abs(line["ms_per_step"] - 2500.0) < 1e-9
    assert line["cpu_baseline"]["value"] == line["value"] and line["e2e"]["value"] == line["value"]
