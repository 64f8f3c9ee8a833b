"""The N > 1 path of the benchmark on CPU: independent replicas, one per
rank, whose job time is the slowest rank's and whose value counts every
rank's member solves (two gloo ranks; the GPU run uses NCCL the same way)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        t_max = bench.max_over_ranks(times[rank], torch.device("cpu"))
        out[rank] = (t_max, bench.replica_value(51, 5, w, t_max))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_take_the_slowest_time_and_count_every_rank(world):
    times = [1.25, 2.5]
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        t_max, value = out[r]
        assert t_max == max(times)
        assert value == pytest.approx(world * 51 * 5 / max(times))


def test_single_rank_defaults():
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.replica_value(51, 2, 1, 2.0) == 51.0
