"""bench.py's multi-GPU form is independent replicas (the path shards into no collective): the
job's time is the slowest rank's and its rate counts every rank's units.  Checked here with two
gloo ranks on the CPU; the reference arm's other ranks exit without work."""
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


RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo")
ms = [12.5, 20.0][rank]
worst = bench.max_over_ranks(ms, world, "cpu")
rate = bench.replica_rate(1000, world, worst)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "worst": worst, "rate": rate}))
"""


def _launch(script_args, world, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable] + script_args, env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_two_gloo_ranks_take_the_slowest_time():
    pytest.importorskip("torch.distributed")
    outs = _launch(["-c", RANK_SCRIPT], 2)
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["worst"] == 20.0                    # the max over both ranks, on every rank
        assert r["rate"] == pytest.approx(2 * 1000 / 0.020)


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun the oracle arm runs on rank 0; rank 1 exits 0 without work or output."""
    outs = _launch(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", "--gpus", "2"], 2)
    lines = [o.strip().splitlines() for o in outs]
    assert lines[1] == []
    line = json.loads(lines[0][-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
