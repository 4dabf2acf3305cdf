"""The multi-rank bench logic on CPU: two gloo ranks on 127.0.0.1.

bench.py runs one independent replica of the window step per GPU (the path
has no exchange step, so there is no data-path collective); what crosses
ranks is the barrier and the maximum of the per-rank timings, from which the
whole-job rate is formed.  Those are checked here with world_size 2.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["GS_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % os.environ["GS_PORT"],
                        rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
world, rank, local = bench.dist_env()
mine = [10.0 + 5.0 * rank, 20.0 - 3.0 * rank]
dist.barrier()
mx = bench.max_over_ranks(mine, world, device="cpu")
rate = bench.whole_job_rate(world, 50, mx[0])
print(json.dumps({"rank": rank, "world": world, "max": mx, "rate": rate}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_replica():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), GS_PORT=str(port),
                   GS_ROOT=ROOT, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["world"] == 2
        assert o["max"] == [15.0, 20.0]           # rank 1's first, rank 0's second
        assert abs(o["rate"] - 2 * 50 / 0.015) < 1e-6   # both replicas' steps over the slowest time


def test_one_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, device="cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(1, 10, 20.0) == 500.0
