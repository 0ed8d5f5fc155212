"""Multi-rank path on CPU: two gloo ranks run independent replicas; the
slowest rank's time sets the whole-job throughput, and only rank 0 reports."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_2210_17509_gb300.replicas import Replicas
    R = Replicas("gloo")
    R.barrier()
    ms = R.max_over_ranks(10.0 + 5.0 * rank)         # rank 1 is the slow one
    rate = R.job_rate(1000.0, ms)
    out.put((rank, ms, rate, R.is_root))
    R.barrier()
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, root in res:
        assert ms == 15.0
        assert rate == pytest.approx(2 * 1000.0 / 15e-3)
        assert root == (rank == 0)


def test_single_process_needs_no_process_group():
    from paper_2210_17509_gb300.replicas import Replicas
    R = Replicas("gloo")
    assert R.world == 1 and R.max_over_ranks(3.5) == 3.5 and R.is_root
