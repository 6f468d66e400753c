"""The multi-rank path of bench.py on CPU: 2 gloo ranks, independent work, max-over-ranks timing."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    vals = bench.reduce_max([1.0 + rank, 10.0 - rank, 3.0], world)
    out.put((rank, vals, bench.weak_scaling_value(1e9, world, vals[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, vals, value in res:
        assert vals == [2.0, 10.0, 3.0]
        assert value == pytest.approx(2 * 1e9 / 2e-3 / 1e9)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.weak_scaling_value(2e9, 1, 1000.0) == pytest.approx(2.0)
