"""bench.py's multi-rank bookkeeping (one independent replica per rank, no
data-path collective): the timing is the maximum over ranks and the value is
the whole job's cell-updates over that time.  Two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 * (rank + 1)           # rank 1 is the slower one
        slow = bench.slowest_rank_ms(ms, world, "cpu")
        q.put((rank, slow, bench.whole_job_rate(1000, 5, world, slow)))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, rate in res:
        assert slow == 20.0
        assert rate == pytest.approx(2 * 1000 * 5 / 0.020 / 1e9)
