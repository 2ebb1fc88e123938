"""The multi-process path of bench.py on CPU: two ranks over gloo.

Quartets are independent, so N GPUs run N replicas; the only collective is the max over
ranks of the timing.  These tests run that collective, the barrier and the reference arm's
rank handling with world size 2 on the host."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank), "LX_BENCH_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import bench
    r, local, w = bench.dist_setup(world)
    try:
        bench.barrier(w)
        # each rank reports its own step time; every rank must see the largest
        got = bench.reduce_max(10.0 + 5.0 * r, w)
        bench.barrier(w)
        q.put((r, local, w, got))
    finally:
        dist.destroy_process_group()


def test_timing_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    assert [x[0] for x in res] == [0, 1]
    assert all(x[2] == 2 for x in res)
    assert all(x[3] == 15.0 for x in res)


def test_reference_arm_prints_once_under_torchrun():
    # rank 0 times the CPU oracle and prints one JSON line; rank 1 exits 0 without work
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--nquartet", "64"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
