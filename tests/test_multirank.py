"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1) reduce their
timed regions to the slowest rank's and report whole-job throughput, and the
reference arm runs on rank 0 only.  Replicas share no data, so this reduction
is the only collective of the job."""
import json
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


WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
elapsed = [3.0, 5.0][rank]
t = bench.max_over_ranks(elapsed, world)
print(json.dumps({{"rank": rank, "t_max": t, "value": bench.job_throughput(world, 4, t)}}))
dist.destroy_process_group()
"""


def _launch(code, world=2, extra=()):
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()), WORLD_SIZE=str(world))
    procs = []
    for r in range(world):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, *code], env=e, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_two_gloo_ranks_take_the_slowest_time():
    outs = _launch(["-c", WORKER.format(root=ROOT)])
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["t_max"] == 5.0                  # both ranks see the slowest rank's time
        assert r["value"] == pytest.approx(2 * 4 / 5.0)   # whole job: 2 ranks x 4 units in 5 s


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm's rank 0 prints the one JSON line and the
    other ranks exit 0 without work (the smallest workload keeps this quick)."""
    outs = _launch(["bench.py", "--impl", "reference", "--workload", "poisson2d_64", "--steps", "1",
                    "--warmup", "3", "--gpus", "2"])
    lines0 = [l for l in outs[0].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and json.loads(lines0[0])["impl"] == "reference"
    assert not [l for l in outs[1].splitlines() if l.startswith("{")]
