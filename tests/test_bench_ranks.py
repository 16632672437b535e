"""The bench's multi-GPU path is N independent replicas: each rank times its
own run, the job time is the maximum over ranks (all_reduce MAX), and the
value is the total node updates over that time.  Checked with two gloo ranks
on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(torch, 1.0 + rank, "cpu")
    v = bench.replica_value(1000, 10, world, t)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_value_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]
    assert all(abs(o[2] - 2 * 1000 * 10 / 2.0 / 1e6) < 1e-12 for o in out)


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(torch, 3.5, "cpu") == 3.5
    assert bench.replica_value(16777216, 1000, 1, 0.5) == pytest.approx(33554.432)
