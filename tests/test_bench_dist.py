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


def test_oracle_replicas_on_threads_agree_with_one_oracle_call():
    """The CPU baseline runs one oracle replica per core on threads; every
    replica's state after two steps equals the oracle run alone on the same
    input (the oracle keeps no shared state between calls)."""
    import numpy as np

    import bench
    from oracle import oracle as O
    r = bench.OracleReplicas(12, 3)
    p0, c = r.p[0].copy(), r.c
    r.step()
    r.step()
    r.close()
    ref = O.step(O.step(p0, c, O.CEC, 0), c, O.CEC, 1)
    for p in r.p:
        assert np.array_equal(p, ref)


def test_reference_arm_prints_one_line_with_its_core_count():
    import json
    import subprocess
    import sys

    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["cores"] == bench.host_cores()
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_other_ranks_exit_without_work():
    """Under a multi-rank launch only rank 0 times the oracle; rank 1 exits 0
    and prints nothing."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT="29999")
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=120, cwd=root,
                         env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
