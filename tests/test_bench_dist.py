"""The multi-rank plumbing of bench.py on CPU: two gloo ranks (the GPU arm
uses the same calls over NCCL, one replica per GPU).  The whole-job number is
the units of all ranks over the slowest rank's time, and the reference arm
prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


WORKER = r"""
import json, os, sys, types
sys.path.insert(0, sys.argv[1])
import bench
import torch.distributed as dist
rank, world, local = bench.dist_init(types.SimpleNamespace(impl="reference"))
ms, value = bench.replica_throughput([10.0 + 5.0 * rank, 20.0], 1000, world)
bench.barrier(world)
print(json.dumps({"rank": rank, "world": world, "ms": ms, "value": value}), flush=True)
dist.destroy_process_group()
"""


def _launch(code, world, extra=()):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE=str(world),
                   LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *extra], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_replica_throughput_takes_the_slowest_rank():
    pytest.importorskip("torch")
    outs = _launch(WORKER, 2)
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for d in lines:
        assert d["world"] == 2
        # rank 1 is slower: (15 + 20) ms for 2 steps; 2 ranks x 1000 units x 2 steps
        assert d["ms"] == pytest.approx(17.5)
        assert d["value"] == pytest.approx(2 * 1000 * 2 / 35e-3)


REF = r"""
import os, runpy, sys
root = sys.argv[1]
sys.path.insert(0, root)
sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
runpy.run_path(os.path.join(root, "bench.py"), run_name="__main__")
"""


def test_reference_arm_prints_on_rank0_only():
    """Each rank of the reference arm under torchrun: rank 0 times the oracle
    sample and prints the JSON line, rank 1 exits 0 without work."""
    pytest.importorskip("torch")
    outs = _launch(REF, 2)
    printed = [o.strip().splitlines() for o in outs]
    assert len(printed[1]) == 0
    d = json.loads(printed[0][-1])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
