"""The N-GPU bench path runs replicas: one process per GPU, each factoring its own matrix, with
no collective on the data path.  Its host logic is checked with two gloo ranks on CPU:
  * the job's time is its slowest rank's (max over ranks);
  * the whole-job rate counts the work of every rank over that time;
  * every rank draws its own matrix (distinct seeds);
  * under torchrun only rank 0 runs and prints the reference arm.
"""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        dist.barrier()
        ms = [10.0, 14.0][rank]                       # rank 1 is the slow one
        t = bench.max_over_ranks(ms, world, torch.device("cpu"))
        rate = bench.job_rate(100.0, world, t)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(1000, rank))
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, t, rate, seeds, None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, None, None, repr(e)))


def test_two_gloo_ranks_aggregate_like_the_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    try:
        res = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.kill()
    for rank, t, rate, seeds, err in res:
        assert err is None, (rank, err)
        assert t == 14.0                              # the slowest rank's time
        assert rate == pytest.approx(2 * 100.0 / 0.014)
        assert len(set(seeds)) == 2                   # each replica draws its own matrix
    assert [r[0] for r in res] == [0, 1]


def test_single_rank_helpers_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.job_rate(10.0, 1, 1000.0) == pytest.approx(10.0)
    assert bench.replica_seed(7, 0) == 7


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.main() == 0
    assert buf.getvalue() == ""
