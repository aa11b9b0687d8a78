"""The multi-GPU path (replicas: one process per GPU, views split across ranks, no data-path
exchange) on CPU with world size 2 over gloo: the ranks' view cycles partition the views, every
rank does the same work per step, the job time is the slowest rank's, and the whole-job rate is
the units of all ranks over that time."""
import os
import socket

import pytest

from paper_2411_14974_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, views, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = replicas.dist_env()
        mine = replicas.views_for_rank(views, r, ws)
        gathered = [None] * ws
        dist.all_gather_object(gathered, mine)
        replicas.barrier()
        slowest = replicas.max_over_ranks(times[r])
        out.put((r, ws, local, gathered, slowest, replicas.job_throughput(100.0, ws, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_views_and_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    views = ["v0", "v1", "v2", "v3", "v4", "v5"]
    times = [12.5, 20.0]  # ms per rank
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, views, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ws, local, gathered, slowest, rate in res:
        assert ws == 2 and local == r
        a, b = gathered
        assert len(a) == len(b) == len(views)          # equal work per step
        assert set(a) == {"v0", "v2", "v4"} and set(b) == {"v1", "v3", "v5"}  # disjoint, covering
        assert slowest == 20.0                           # the job takes its slowest rank's time
        assert rate == pytest.approx(2 * 100.0 / 0.020)  # both ranks' units over that time


def test_single_process_helpers():
    assert replicas.views_for_rank([1, 2, 3], 0, 1) == [1, 2, 3]
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(10.0, 1, 0.0) == 0.0
    with pytest.raises(ValueError):
        replicas.views_for_rank([1, 2], 2, 2)
