"""The bench's multi-GPU arithmetic on CPU: two gloo ranks, each with its own map
time and interaction count; the whole-job figures are the max time and the sum of
interactions (independent maps, weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, n = bench.reduce_over_ranks(dist, "cpu", 1.0 + rank, 10 ** 12 * (rank + 1))
    out[rank] = (t, n)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = tmp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, n = out[r]
        assert t == pytest.approx(2.0)
        assert n == pytest.approx(3e12)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, "cpu", 1.5, 7) == (1.5, 7)
