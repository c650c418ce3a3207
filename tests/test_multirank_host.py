"""The N > 1 path of bench.py on CPU with world-size-2 gloo ranks: the step time
is the maximum over ranks; with replicas the value counts every rank's pixels
(no data-path collective), with the tile split the ranks share one frame's
pixels (no GPU)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    value, t = bench.aggregate(local_ms, pixels_per_rank=1_000_000, steps=10, world=world, dist=dist, device="cpu")
    # the tile split: the ranks share one frame (strong scaling)
    shared, ts = bench.aggregate(local_ms, pixels_per_rank=1_000_000, steps=10, world=world, dist=dist,
                                 device="cpu", shared=True)
    q.put((rank, value, t, shared, ts))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t, shared, ts in res:
        assert t == pytest.approx(150.0) and ts == pytest.approx(150.0)
        assert value == pytest.approx(2 * 1_000_000 * 10 / 0.150 / 1e6)
        assert shared == pytest.approx(1_000_000 * 10 / 0.150 / 1e6)


def test_single_rank_aggregate_is_local():
    import bench
    value, t = bench.aggregate(200.0, 1_228_800, 20, 1)
    assert t == 200.0 and value == pytest.approx(1_228_800 * 20 / 0.2 / 1e6)
