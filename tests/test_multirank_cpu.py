"""The multi-GPU path of bench.py is replicas only: every rank sweeps its own
MERA and the only collectives are a barrier and the max over ranks of the
timed region.  This exercises that host logic with two gloo ranks on the CPU
(no GPU): each rank reports a different time, both must see the slowest, and
the job throughput is world x steps / slowest time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench._dist()
        assert (w, r, local) == (world, rank, rank)
        mine = 100.0 + 50.0 * rank  # rank 1 is the slowest
        torch.distributed.barrier()
        slowest = bench._max_over_ranks(mine, "cpu")
        value = bench._job_throughput(w, 3, slowest)
        out.put((rank, slowest, value))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in res:
        assert slowest == 150.0
        assert value == pytest.approx(2 * 3 / 0.150)


def test_single_process_needs_no_group():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    assert bench._max_over_ranks(12.5, "cpu") == 12.5
    assert bench._job_throughput(1, 4, 2000.0) == pytest.approx(2.0)
