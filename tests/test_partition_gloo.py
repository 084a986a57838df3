"""The batched form shards across GPUs with no exchange on the data path: each rank factors its
LPT share of the one batch (paper_1804_05138_gb300.partition).  Checked on CPU:
  * every matrix of the 512-matrix batch is assigned exactly once, for 1..8 ranks;
  * the ranks' counted-flop loads differ by at most the largest single matrix's cost;
  * with two gloo ranks, each factoring its share of a small uneven batch (the CPU oracle stands
    in for the batched kernel, which needs a GPU), the gathered results cover every matrix once
    and every rank equals its k; the job's flops are the sum over ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1804_05138_gb300 import inputs, partition  # noqa: E402


def _cost(m, n, k, b=64, p=8):
    l = b + p
    return 2.0 * l * m * n + 4.0 * m * n * k - 2.0 * (m + n) * k * k + 4.0 * k ** 3 / 3.0


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_lpt_partition_covers_the_batch_and_balances(world):
    shapes = inputs.batched_shapes(512, seed=0)
    costs = [_cost(m, n, k) for m, n, k in shapes]
    parts = partition.lpt_partition(costs, world)
    assert len(parts) == world
    flat = sorted(i for part in parts for i in part)
    assert flat == list(range(len(shapes)))
    loads = partition.rank_loads(costs, parts)
    assert max(loads) - min(loads) <= max(costs)
    assert sum(loads) == pytest.approx(sum(costs))


def test_lpt_partition_small_cases():
    assert partition.lpt_partition([], 3) == [[], [], []]
    assert partition.lpt_partition([5.0], 2) == [[0], []]
    # classic LPT example: costs 7,6,5,4 on two ranks -> {7,4}, {6,5}
    parts = partition.lpt_partition([4.0, 7.0, 5.0, 6.0], 2)
    assert parts == [[1, 0], [3, 2]]
    with pytest.raises(ValueError):
        partition.lpt_partition([1.0], 0)


SMALL = [(60, 40, 12), (90, 30, 20), (45, 45, 9), (120, 64, 30), (33, 20, 20), (70, 50, 16), (100, 80, 25)]


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    try:
        import torch
        import torch.distributed as dist
        import bench
        from oracle import oracle
        from paper_1804_05138_gb300 import inputs as inp, partition as part
        dist.init_process_group("gloo", rank=rank, world_size=world)
        b, p = 8, 4
        costs = [_cost(m, n, k, b, p) for m, n, k in SMALL]
        mine = part.lpt_partition(costs, world)[rank]
        Om = oracle.omega(b + p, max(m for m, _, _ in SMALL), seed=0)
        done = []
        for i in mine:
            m, n, k = SMALL[i]
            A = inp.spectrum_matrix(m, n, inp.sigma_exp_decay(min(m, n), 0.1 * n), 1000 + 2 * i, 1001 + 2 * i)
            res = oracle.rqrcp(A, k, b, p, np.ascontiguousarray(Om[:, :m]))
            done.append((i, int(res.rank), k))
        F = sum(costs[i] for i in mine)
        F_job = bench.sum_over_ranks(F, world, torch.device("cpu"))
        gathered = [None] * world
        dist.all_gather_object(gathered, done)
        dist.destroy_process_group()
        q.put((rank, gathered, F_job, sum(costs), None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, None, None, repr(e)))


def test_two_gloo_ranks_factor_disjoint_shares():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.kill()
    for rank, gathered, F_job, F_all, err in res:
        assert err is None, (rank, err)
        flat = [t for per in gathered for t in per]
        assert sorted(i for i, _, _ in flat) == list(range(len(SMALL)))   # each matrix once
        assert all(r == k for _, r, k in flat)                             # rank equals k
        assert all(len(per) > 0 for per in gathered)                       # both ranks worked
        assert F_job == pytest.approx(F_all)                               # job flops = sum over ranks
