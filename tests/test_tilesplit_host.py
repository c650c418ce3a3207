"""Host side of the tile-split step on CPU with world-size-2 gloo ranks.

Each rank takes its tiles from geer_tile_owners (a host-only call of the
library), renders (here: the oracle's FP64 gradient of its own pixels) and the
step's one exchange, an all-reduce sum, gives every rank the full gradient. The
test checks that the partition covers every tile and every pixel exactly once,
that the parts are balanced, and that the reduced gradient equals the oracle's
gradient of the whole image."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2505_24053_gb300 import workloads as wl

CAMS = [wl.Camera(wl.EQUIDISTANT, 48, 40, math.radians(190)),
        wl.Camera(wl.PINHOLE, 35, 24, math.radians(60), R_cw=wl.pose(wl.rot_y(0.5), (0.2, 0.0, -0.3))[0],
                  t_cw=wl.pose(wl.rot_y(0.5), (0.2, 0.0, -0.3))[1])]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _scene():
    return wl.cube_scene(96, 23, 1)


def _weights(cam, k):
    return np.random.default_rng(50 + k).normal(0, 1, (cam.pixels, 3))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as orc
        from paper_2505_24053_gb300 import geer, tilesplit
        orc.build()
        tiles = torch.as_tensor((geer.tile_owners(CAMS, world) == rank).astype(np.int32))
        pix = torch.as_tensor((tilesplit.pixel_owners(CAMS, world) == rank).astype(np.int32))
        all_tiles = [torch.zeros_like(tiles) for _ in range(world)]
        all_pix = [torch.zeros_like(pix) for _ in range(world)]
        dist.all_gather(all_tiles, tiles)
        dist.all_gather(all_pix, pix)
        # this rank's gradient: the oracle's FP64 gradient of sum(w * C) over its own pixels
        scene = _scene()
        parts, off = [], 0
        for k, cam in enumerate(CAMS):
            own = pix.numpy()[off:off + cam.pixels].astype(bool)
            off += cam.pixels
            allpix = wl.all_pixels(cam)
            g = orc.render_grad(scene, cam, allpix[own], _weights(cam, k)[own])
            parts.append(np.concatenate([g[n].ravel() for n in ("mean", "scale", "quat", "opacity", "sh")]))
        flat = torch.as_tensor(np.sum(parts, axis=0))
        tilesplit.reduce_sum(flat, None, world)
        q.put((rank, torch.stack(all_tiles).numpy(), torch.stack(all_pix).numpy(), flat.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_tile_split_partition_and_gradient_reduction_on_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    tiles, pix = res[0][1], res[0][2]
    assert np.array_equal(tiles.sum(axis=0), np.ones(tiles.shape[1]))  # every tile owned once
    assert np.array_equal(pix.sum(axis=0), np.ones(pix.shape[1]))      # every pixel owned once
    assert abs(int(tiles[0].sum()) - int(tiles[1].sum())) <= len(CAMS)  # checkerboard halves
    # every rank ends with the same reduced gradient, equal to the whole image's
    from oracle import oracle as orc
    orc.build()
    scene = _scene()
    full = 0
    for k, cam in enumerate(CAMS):
        g = orc.render_grad(scene, cam, wl.all_pixels(cam), _weights(cam, k))
        full = full + np.concatenate([g[n].ravel() for n in ("mean", "scale", "quat", "opacity", "sh")])
    for rank, _, _, flat in res:
        assert np.allclose(flat, full, rtol=1e-10, atol=1e-12 * np.abs(full).max()), rank
        assert np.abs(flat - res[0][3]).max() == 0.0
    # the split is not trivial: each rank's own part differs from the full gradient
    assert np.abs(full).max() > 0


def test_tile_owners_balance_and_argument_errors():
    from paper_2505_24053_gb300 import geer
    cam = wl.config_cameras(3)[0]  # 1280 x 960: 80 x 60 tiles
    for n in (2, 3, 4, 8):
        own = geer.tile_owners([cam], n)
        counts = np.bincount(own, minlength=n)
        assert counts.sum() == 80 * 60 and counts.min() >= 0.97 * counts.mean()
        # each part has tiles in every 16 x 16 block of tiles: no region is one part's alone
        grid = own.reshape(60, 80)
        for by in range(0, 48, 16):
            for bx in range(0, 64, 16):
                assert len(np.unique(grid[by:by + 16, bx:bx + 16])) == n
    with pytest.raises(geer.GeerError):
        geer.tile_owners([cam], 0)
