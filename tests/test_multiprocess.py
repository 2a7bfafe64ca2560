"""The multi-process (N > 1) host logic of bench.py on CPU with gloo ranks.

The single-problem solve does not shard ("replicas only"): with N ranks every
rank runs its own replica, the ranks meet at a barrier around the timed
region, the step time is the maximum over ranks and rank 0 alone prints the
JSON line.  These tests check that logic with world size 2 on the CPU: the
process-group set-up from the torchrun environment, the barrier, the
max-over-ranks reduction, and the reference arm under torchrun (rank 0
prints one line, the other rank exits 0 without output).
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_init()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(ws)
    # every rank reports a different step time; all must agree on the maximum
    v = bench.max_over_ranks(ws, 10.0 + 5.0 * rank)
    out.put((rank, v))
    dist.destroy_process_group()


def test_dist_init_barrier_and_max_over_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(world))
    assert got == [(0, 15.0), (1, 15.0)]


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--workload", "cfg2", "--steps", "1", "--warmup", "0",
           "--ref-rotations", "2000"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
