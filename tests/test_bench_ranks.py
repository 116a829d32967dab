"""The benchmark's multi-rank logic on CPU: two gloo ranks with different
step times agree on the slowest one, the aggregate rate counts every rank's
units, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
        ref = bench.run_reference(None, rank, world) if rank > 0 else "rank0"
        out.put((rank, t, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[1][2] is None       # the reference arm prints on rank 0 only


def test_aggregate_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_rate(1000, 1, 500.0) == pytest.approx(2000.0)
    assert bench.aggregate_rate(1000, 4, 500.0) == pytest.approx(8000.0)
    assert bench.max_over_ranks(7.5, 1, None) == 7.5
