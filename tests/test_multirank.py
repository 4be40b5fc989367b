"""Host logic of several ranks on CPU (world size 2): the bench's seed split, max-over-ranks timing
and whole-job throughput over a gloo process group, and the reference arm under
torch.distributed.run (rank 0 alone prints one line; the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seeds = [bench.mock_seed(rank, ph, i) for ph in range(6) for i in range(100)]
        every = [None] * world
        dist.all_gather_object(every, seeds)
        ms = 10.0 + 5.0 * rank                      # the slower rank decides the job's time
        mx = bench.reduce_max(ms, dist)
        value = bench.job_value(1000, world, mx)
        if rank == 0:
            out.put({"seeds": every, "max": mx, "value": value})
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_seeds_and_reduce_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    a, b = (set(x) for x in res["seeds"])
    assert len(a) == 600 and len(b) == 600 and not (a & b)      # disjoint across ranks and phases
    assert res["max"] == 15.0
    assert res["value"] == pytest.approx(1000 * 2 / 0.015)


def test_reference_arm_under_torchrun_prints_once():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
