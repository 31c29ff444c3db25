"""The multi-process (replicas) path of bench.py on CPU, world size 2, gloo.

The single-GPU path has no exchange step, so N GPUs run N independent
replicas; the ranks meet only for the barrier around the timed region and
the max (time) / sum (work) over ranks. These tests run those helpers and
the reference arm's rank handling in two gloo processes on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local = bench.dist_env()
    dist = bench.init_dist(ws)
    bench.barrier(dist)
    mx = bench.reduce_max(dist, float(rank + 1) * 1.5)
    sm = bench.reduce_sum(dist, float(rank + 1))
    # each replica integrates its own seeded workload (weak scaling)
    from paper_1205_2288_gb300 import inputs
    m, rr, v = inputs.plummer(64, bench.SEED + r)
    bench.barrier(dist)
    dist.destroy_process_group()
    out.put((r, ws, local, mx, sm, float(rr[0, 0])))


def test_barrier_and_reductions_over_two_ranks():
    port = free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(k, port, q))
             for k in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [x[0] for x in res] == [0, 1]
    for r, ws, local, mx, sm, _ in res:
        assert ws == 2 and local == r
        assert mx == 3.0 and sm == 3.0
    assert res[0][5] != res[1][5]   # different seeds per replica


@pytest.mark.slow
def test_reference_arm_prints_once_under_torchrun():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
           "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
