"""The multi-process path of bench.py on CPU (gloo, world size 2): one process
per rank, independent replicas, barrier and max-over-ranks timing, a single
JSON line from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env():
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    env["OMP_NUM_THREADS"] = "2"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    return env


def test_dist_barrier_and_max_over_ranks_gloo():
    """Each rank reports a different elapsed time; every rank sees the maximum."""
    script = r'''
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import bench
d = bench.Dist()
assert d.world == 2
d.barrier()
m = d.max(1.5 + d.rank)
print(json.dumps({"rank": d.rank, "max": m}), flush=True)
d.close()
'''
    port = _free_port()
    procs = []
    for rank in range(2):
        env = _env()
        env.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": "2",
                    "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "ROOT": ROOT})
        procs.append(subprocess.Popen([sys.executable, "-c", script], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    vals = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    assert sorted(v["rank"] for v in vals) == [0, 1]
    assert all(v["max"] == 2.5 for v in vals)


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` launched by torchrun with 2 ranks: rank 0
    alone times the oracle and prints one line; the other rank exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1", "--edge", "32"]
    out = subprocess.run(cmd, cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
