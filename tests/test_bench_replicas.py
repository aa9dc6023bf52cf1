"""The bench's multi-GPU path is replicas only (the FD-CGKS step of one grid
does not shard): each rank advances its own copy, and the job's rate is the
units of all ranks over the slowest rank's time.  These tests run that host
logic as two gloo ranks on the CPU (barrier, max over ranks, the rate, and
the reference arm printing from rank 0 only)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys, time
sys.path.insert(0, os.environ["BENCH_ROOT"])
import bench
world, rank, local = bench.dist_setup(None, backend="gloo")
bench.barrier(world)
el = 0.1 * (rank + 1)                         # rank 1 is the slower replica
rate, el_max = bench.replica_rate(1000.0, el, world)
print(json.dumps({"rank": rank, "world": world, "rate": rate, "el_max": el_max}), flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(code_or_args, world=2, timeout=240):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), BENCH_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        cmd = [sys.executable, "-c", code_or_args] if isinstance(code_or_args, str) else code_or_args
        procs.append(subprocess.Popen(cmd, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    return outs


def test_replica_rate_takes_the_slowest_rank():
    outs = _launch(WORKER)
    res = []
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
        res.append(json.loads(o.strip().splitlines()[-1]))
    for r in res:
        assert r["world"] == 2
        assert r["el_max"] == pytest.approx(0.2)
        assert r["rate"] == pytest.approx(2 * 1000.0 / 0.2)


def test_reference_arm_prints_on_rank_zero_only():
    outs = _launch([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                    "--warmup", "0"])
    lines = []
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
        lines.append([l for l in o.splitlines() if l.strip().startswith("{")])
    assert len(lines[0]) == 1 and len(lines[1]) == 0
    line = json.loads(lines[0][0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2


def test_oracle_all_cores_leg():
    """The all-cores CPU baseline: one spawned process per core, each running
    its own copy of the bounded oracle sample; the aggregate rate counts every
    copy over the wall time of the concurrent runs."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench\n"
            "r, wall, n = bench.oracle_rate_all_cores(8, 1, ncores=2)\n"
            "print(json.dumps({'rate': r, 'wall': wall, 'n': n}))\n" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["n"] == 2 and res["wall"] > 0
    assert res["rate"] == pytest.approx(2 * 2 * 8 * 8 * 1 / res["wall"], rel=1e-12)
