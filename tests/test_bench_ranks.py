"""The bench's multi-process host logic (no GPU): with WORLD_SIZE = 2, two
gloo ranks join one process group through the same environment torchrun
sets, the barrier passes and the time reported is the maximum over the
ranks, which is what the bench's one JSON line (rank 0) divides the units of
all ranks by."""
import os
import socket

import pytest


def _rank(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import torch.distributed as dist
    ws, r, _ = bench.dist_setup()
    bench.barrier(ws)
    m = bench.max_over_ranks(0.5 + r, ws)   # rank 1 is the slower one
    bench.barrier(ws)
    out.put((r, ws, m))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_report_the_slowest():
    import torch.multiprocessing as mp
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
    assert res == [(0, 2, 1.5), (1, 2, 1.5)]


def test_one_rank_needs_no_process_group():
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        ws, rank, local = bench.dist_setup()
        assert (ws, rank, local) == (1, 0, 0)
        assert bench.max_over_ranks(2.5, ws) == 2.5
    finally:
        os.environ.update(env)
