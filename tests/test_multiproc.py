"""The N > 1 host logic of bench.py (replicas, no data-path collective) on CPU
with world-size-2 gloo process groups: the timed region closes with a
barrier, the job time is the slowest rank's, and the whole-job throughput
counts every replica's units; the reference arm runs on rank 0 alone."""
import contextlib
import io
import json
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local, units, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier_all(world)
        t = bench.max_over_ranks(local[rank], world, device="cpu")
        v = bench.job_throughput(units, world, t)
        bench.barrier_all(world)
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_throughput_counts_all_replicas():
    world, units = 2, 1_310_720 * 10
    local = [0.412, 0.537]                     # per-rank timed-region seconds
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, local, units, q))
             for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, t, v in res:
        assert t == max(local), rank
        assert v == pytest.approx(world * units / max(local), rel=1e-15)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.barrier_all(1)
    assert bench.max_over_ranks(0.25, 1) == 0.25
    assert bench.job_throughput(100, 1, 0.5) == 200.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun every rank runs `bench.py --impl reference`; ranks other
    than 0 return at once, print nothing and open no process group."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    called = []
    monkeypatch.setattr(bench, "run_reference", lambda args: called.append(args) or {})
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.main()
    assert out.getvalue() == "" and not called
    monkeypatch.setenv("RANK", "0")
    with contextlib.redirect_stdout(out):
        bench.main()
    assert len(called) == 1 and json.loads(out.getvalue().strip().splitlines()[-1]) == {}
