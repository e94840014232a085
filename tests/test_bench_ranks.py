"""The multi-rank path of the benchmark on CPU: world-size-2 gloo groups
(one process per rank, as torchrun starts them) reduce the step time to the
maximum over ranks and scale the whole-job throughput by the rank count."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]
        w, r, loc = bench._dist()
        q.put((rank, bench.max_over_ranks(ms), (w, r, loc)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, (w, r, loc) in res:
        assert v == 20.0
        assert (w, r, loc) == (world, rank, rank)


def test_max_over_ranks_without_a_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
