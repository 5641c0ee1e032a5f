"""The multi-GPU path of bench.py is replicas only: the sole collectives are the timing barrier and
the max of the elapsed time over ranks.  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench.barrier()
    out[rank] = bench.aggregate_max(1.5 + rank)  # elapsed of the slowest rank
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        assert dict(out) == {0: 2.5, 1: 2.5}


def test_single_process_aggregate_is_identity():
    import bench

    assert bench.aggregate_max(3.25) == 3.25


def test_select_steps_holds_the_growth_steps():
    import bench

    growth = (33, 34, 35, 36)
    # the driver's sample: 20 of the steps after 5 warm-up steps, growth steps always in it
    t = bench.select_steps(50, 5, 20, growth)
    assert len(t) == 20 and all(s - 1 in t for s in growth)
    assert t == sorted(t) and t[0] >= 5 and t[-1] <= 49
    # a budget covering the range times all of it
    assert bench.select_steps(50, 3, 47, growth) == list(range(3, 50))
    # no growth steps: one timed step is the first after the warm-up
    assert bench.select_steps(50, 3, 1, ()) == [3]
    # fewer steps than growth steps: the first ones of them
    assert bench.select_steps(50, 5, 2, growth) == [32, 33]
