"""The multi-GPU path of bench.py is replicas (the solver does not shard:
every rank solves its own problem on its own GPU): the host logic of that path
on CPU ranks under gloo, world size 2 -- the max over ranks that times the job,
the ranks' distinct problems, and the reference arm's ranks other than 0
exiting without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); ws = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=ws)
vals = [3.5, 11.25]
got = bench.max_over_ranks(vals[rank], ws, "cpu")
dist.barrier()
seed = bench.replica_seed(rank)
dist.destroy_process_group()
print("RESULT" + json.dumps({"rank": rank, "max": got, "seed": seed}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_replica_seeds_gloo():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads([x for x in out.splitlines() if x.startswith("RESULT")][-1][6:]))
    assert [o["max"] for o in outs] == [11.25, 11.25]
    assert len({o["seed"] for o in outs}) == 2


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, 1, "cpu") == 7.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
