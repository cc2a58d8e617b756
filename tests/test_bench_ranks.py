"""Multi-rank logic of bench.py on CPU: two gloo ranks reduce the timed region
to the slowest rank's time and the sum of certified solves (weak scaling,
no collective on the data path)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        secs, ok = bench.job_totals(w, 1.0 + 0.5 * r, 4000 + r, torch.device("cpu"))
        q.put((r, w, local, secs, ok))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_time_and_solves():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rr, w, local, secs, ok) in enumerate(got):
        assert (rr, w, local) == (r, 2, r)
        assert secs == pytest.approx(1.5)   # the slowest rank
        assert ok == 4000 + 4001            # certified solves of both ranks


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(1, 2.0, 17, None) == (2.0, 17)
