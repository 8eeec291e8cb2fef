"""The benchmark's multi-rank bookkeeping on CPU: two gloo ranks on 127.0.0.1.

`bench.py --gpus N` runs one independent replica of the solve per GPU (the single-problem
workload has no exchange step); the whole-job rate is every rank's steps over the slowest
rank's time.  These tests run that reduction with world size 2 over gloo, and the
reference arm's rule that only rank 0 prints.
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


def _rank_main(rank, world, port, local_ms, steps, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rate, ms_step = bench.job_rate(local_ms[rank], steps, world, dist, "cpu")
        out.put((rank, rate, ms_step))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    world, steps = 2, 5
    local_ms = [100.0, 250.0]                         # rank 1 is the slower one
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, local_ms, steps, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms_step in res:
        assert ms_step == pytest.approx(250.0 / steps)          # both ranks see the max
        assert rate == pytest.approx(world * steps / 0.250)     # every rank's steps / slowest time


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    rate, ms_step = bench.job_rate(400.0, 4, 1)
    assert ms_step == pytest.approx(100.0)
    assert rate == pytest.approx(10.0)


def test_reference_arm_prints_on_rank_0_only(tmp_path):
    """Under torchrun the reference arm's rank 1 exits 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "args = type('A', (), {'workload': 'c3_bf16_n262144', 'ref_rows': 256, 'warmup': 0, 'steps': 1})(); "
            "bench.run_reference(args, 1, 2)" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
    for line in r.stdout.splitlines():      # nothing that parses as a result line
        with pytest.raises(json.JSONDecodeError):
            json.loads(line)
