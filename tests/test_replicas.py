"""Multi-GPU is replicas only (every rank codes its own copy of the workload, no data-path
collective): the host-side aggregation of bench.py over world_size 2 gloo ranks on the CPU, the
largest time over ranks and the whole-job throughput every rank reports."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w = bench._dist()
        ms = bench.max_over_ranks(times[rank], "cpu")
        q.put((rank, r, w, ms, bench.job_throughput(w, 1 << 24, ms)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(12.5, 30.0), (41.0, 7.25)])
def test_two_gloo_ranks_max_time_and_job_throughput(times):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max(times)
    for rank, (r, rr, w, ms, value) in enumerate(out):
        assert r == rr == rank and w == 2
        assert ms == slowest
        assert value == pytest.approx(2 * (1 << 24) / 1e6 / (slowest / 1e3))


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 10 ** 6, 1000.0) == pytest.approx(1.0)
