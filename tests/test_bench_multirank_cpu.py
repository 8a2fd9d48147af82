"""bench.py's multi-rank logic on CPU: two gloo ranks, max-over-ranks timing, whole-job value."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, %(root)r)
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
ms = bench.aggregate(100.0 + 50.0 * rank, world, dist)
val = bench.job_value(1_000_000_000, world, ms)
print("rank", rank, ms, round(val, 6), flush=True)
dist.destroy_process_group()
"""


def _launch(code, world, port):
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_max_over_ranks_and_job_value():
    outs = _launch(WORKER % {"root": ROOT}, 2, 29511)
    for rank, o in enumerate(outs):
        parts = o.split()
        assert parts[0] == "rank" and int(parts[1]) == rank
        assert float(parts[2]) == 150.0                  # the slower rank's time, on every rank
        assert float(parts[3]) == pytest.approx(2 * 1.0 / 0.150)   # two replicas of 1e9 updates in 150 ms


def test_reference_arm_prints_on_rank_zero_only():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import bench\n"
            "sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', '--warmup', '0']\n"
            "bench.N_SIDE = 64\n"
            "bench.main()\n" % ROOT)
    outs = _launch(code, 2, 29512)
    import json
    line = json.loads(outs[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert outs[1].strip() == ""
