"""Host logic of bench.py under torchrun with two ranks (gloo on CPU).

The benchmark's multi-GPU mode runs independent replicas: every rank reads its
rank from the environment, the timing taken is the maximum over ranks, and only
rank 0 runs and prints the oracle (reference) line."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys, types
sys.path.insert(0, os.environ["BENCH_ROOT"])
import bench
ws, rank, local = bench.dist_init()
mx = bench.max_over_ranks(float(rank + 1) * 0.5, ws)
bench.barrier(ws)
# a rank other than 0 leaves the reference arm without work
args = types.SimpleNamespace(steps=1, warmup=0, gpus=ws)
ran = "skipped"
if rank != 0:
    bench.run_reference(args, ws, rank)
    ran = "returned"
bench.barrier(ws)
print("RESULT " + json.dumps({"ws": ws, "rank": rank, "local": local, "max": mx, "ref": ran}), flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_replicas_max_over_ranks():
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), BENCH_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = []
    for p in procs:
        out, _ = p.communicate(timeout=240)
        assert p.returncode == 0, out
        line = [l for l in out.splitlines() if l.startswith("RESULT ")][-1]
        outs.append(json.loads(line[len("RESULT "):]))
    outs.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in outs] == [0, 1] and all(d["ws"] == 2 for d in outs)
    assert [d["local"] for d in outs] == [0, 1]
    assert all(d["max"] == 1.0 for d in outs)  # max of 0.5 and 1.0 on both ranks
    assert outs[1]["ref"] == "returned"
