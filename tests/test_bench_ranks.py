"""The multi-rank path of bench.py on CPU (gloo, world size 2): the job's
step time is the slowest rank's, the value counts every rank's products, and
the arms that run on one GPU leave the other ranks idle."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % os.environ["MASTER_PORT"],
                        rank=rank, world_size=world)
ms = [3.0, 5.5][rank]
got = bench.max_over_ranks(ms, world, dist, "cpu")
dist.barrier()
print(json.dumps({"rank": rank, "ms": got, "value": bench.whole_job_value(4, world, got)}))
dist.destroy_process_group()
"""


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_max_over_ranks_and_value_gloo():
    port = str(free_port())
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=port)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o.strip().splitlines()[-1])
    import json
    res = [json.loads(x) for x in outs]
    for r in res:
        assert r["ms"] == 5.5  # the slower rank
        assert abs(r["value"] - 2 * 4 / 5.5e-3) < 1e-6


def test_single_gpu_arms_leave_other_ranks_idle():
    for arm in (["--impl", "reference"], ["--workload", "serve"], ["--workload", "product"], ["--workload", "blocked"]):
        env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
        p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + arm + ["--steps", "1", "--warmup", "0"],
                           env=env, capture_output=True, text=True, timeout=120)
        assert p.returncode == 0, p.stderr
        assert p.stdout.strip() == ""
