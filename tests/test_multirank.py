"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
builds its own box from its own seed (independent replicas, no data-path
collective), the slowest rank's time is the job's, and the whole-job rate
counts every rank's cells.  The GPU work itself runs one rank per GPU."""
import os
import socket

import pytest

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.workload(seed_offset=rank, L=24)
        t = bench.max_over_ranks(10.0 + 3.0 * rank, dist)   # rank 1 is the slow one
        dist.barrier()
        q.put((rank, w.n, float(w.pos.sum()), t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_their_own_boxes():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, s0, t0), (r1, n1, s1, t1) = out
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 13.0                      # max over ranks
    assert n0 == n1 and s0 != s1                 # same workload shape, own seeds
    assert bench.max_over_ranks(7.5) == 7.5      # one process: its own time
    # 2 ranks x 13824 cells x 10 steps in 13 ms
    assert bench.job_throughput(2, 13824, 10, 13.0) == pytest.approx(2 * 13824 * 10 / 0.013 / 1e6)
