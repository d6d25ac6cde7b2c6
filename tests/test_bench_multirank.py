"""The bench's multi-GPU path is replicas only: each rank renders its own view and the timed region
is reduced by its maximum over ranks.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [2.0, 3.5][rank]
    m = bench.max_over_ranks(mine)
    agg = bench.aggregate(m, 240, world)
    q.put((rank, m, agg["value"], agg["ms_per_step"]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, value, ms in res:
        assert m == 3.5
        assert value == pytest.approx(2 * 240 / 3.5)
        assert ms == pytest.approx(3.5e3 / 240)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.aggregate(2.0, 100, 1)["value"] == pytest.approx(50.0)
