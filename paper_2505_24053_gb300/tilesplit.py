"""A forward + backward step split by tiles over the ranks of a process group.

Every rank holds the whole scene and the same cameras. The (camera, tile) key
space is partitioned (geer_tile_owners): each rank preprocesses and bins all
Gaussians, renders only its own tiles (geer_set_tile_mask) and runs the
backward's render stage over them (geer_render_bwd_tiles). The render stage's
per-(camera, Gaussian) accumulators are sums over rays, so their sum over the
ranks -- one all-reduce of n_cams x n x 16 f32 -- equals the full image's, and
the preprocess stage (geer_preprocess_bwd) then gives every rank the full
gradient: every rank can take the same optimiser step. A rank's render holds
its own tiles and zeros elsewhere, so the ranks' images sum to the full image.

This is the data-parallel split of the render across GPUs (App. C's two
backward stages with the exchange between them); the paper itself renders on
one GPU. Only the all-reduce crosses processes, through torch.distributed
(NCCL between GPUs, gloo on the CPU), and it reads and writes the accumulators
in the workspace's own device memory.
"""
from __future__ import annotations

import numpy as np
import torch

from . import geer


def pixel_owners(cams, n_parts: int) -> np.ndarray:
    """Owner part of every pixel of the camera set ([total pixels] int32, cameras
    in order, each row-major): the owner of the pixel's tile."""
    owners = geer.tile_owners(cams, n_parts)
    out, t0 = [], 0
    for c in cams:
        tx, ty = (c.width + 15) // 16, (c.height + 15) // 16
        tiles = owners[t0:t0 + tx * ty].reshape(ty, tx)
        out.append(np.repeat(np.repeat(tiles, 16, axis=0), 16, axis=1)[:c.height, :c.width].ravel())
        t0 += tx * ty
    return np.concatenate(out) if out else np.zeros(0, np.int32)


def reduce_sum(t: torch.Tensor, group=None, world: int = 1):
    """Sum a tensor over the ranks in place (the step's one exchange)."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


class TileSplit:
    """This rank's share of a tile-split step over a workspace (geer.Workspace)."""

    def __init__(self, ws: geer.Workspace, rank: int, world: int, group=None):
        if not 0 <= rank < world:
            raise ValueError(f"rank {rank} outside a world of {world}")
        self.ws, self.rank, self.world, self.group = ws, int(rank), int(world), group
        self.set_cameras(ws.cams, upload=False)

    def set_cameras(self, cams, upload: bool = True, stream=None):
        """New camera set (same on every rank): uploads it and this rank's tile mask."""
        if upload:
            self.ws.set_cameras(cams, stream=stream)
        self.cams = list(cams)
        owners = geer.tile_owners(self.cams, self.world)
        self.ws.set_tile_mask(owners == self.rank, stream=stream)
        pix = pixel_owners(self.cams, self.world) == self.rank
        self.pixel_mask = torch.as_tensor(pix.astype(np.float32), device=self.ws.buf.device)

    def masked_target(self, target: torch.Tensor) -> torch.Tensor:
        """The target with zeros outside this rank's pixels: an L1 loss of the
        rank's render against it counts only the rank's pixels (render and target
        are both zero elsewhere, and sign(0) = 0 there), so the ranks' losses sum
        to the full loss."""
        return target.view(-1, 3) * self.pixel_mask[:, None]

    def step(self, g: geer.Gaussians, target_masked: torch.Tensor, rgb: torch.Tensor, dL: torch.Tensor,
             grads: dict, stream=None) -> torch.Tensor:
        """Preprocess, bin, render this rank's tiles, L1 gradient, the render
        stage of the backward, the all-reduce of its accumulators and the
        preprocess stage: grads (written) hold the full gradient on every rank.
        Returns this rank's part of the loss (a device scalar; its sum over the
        ranks is the loss of the full image)."""
        ws = self.ws
        ws.preprocess(g, stream=stream)
        ws.bin_sort(sync=False, stream=stream)
        ws.render_fwd(rgb, None, stream=stream)
        loss, _ = geer.l1_loss_grad(rgb, target_masked, dL, stream=stream)
        ws.render_bwd_tiles(dL, stream=stream)
        acc = ws.grad_accumulators()
        if self.world > 1:
            if stream is not None:
                torch.cuda.current_stream().wait_stream(stream)
            reduce_sum(acc, self.group, self.world)
            if stream is not None:
                stream.wait_stream(torch.cuda.current_stream())
        ws.preprocess_bwd(g, grads, accumulate=False, stream=stream)
        return loss
