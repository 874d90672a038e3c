"""View-sharded multi-view step: the cameras of a step are split across ranks.

Each rank renders its contiguous share of the views (forward and backward, one
batched launch sequence captured in a CUDA graph) over a full replica of the
splat parameters, then one all-reduce (sum) combines the parameter gradients:
the loss of a multi-view step is a sum over views, so its gradient is the sum
of the per-view gradients (Sec. 4.1 trains on one view at a time on one GPU;
splitting the views of a step across GPUs is this library's own design).  The
seven gradient tensors live in one flat buffer, so the exchange is a single
collective: NCCL between GPUs, gloo in the host tests.
"""
from __future__ import annotations

import torch

from .rasterizer import _FIELDS, Gaussians, GraphStep, Rasterizer
from . import hgs as H


def shard_views(pixels, world: int, rank: int):
    """[start, stop) of the views this rank renders: contiguous shares whose pixel
    counts are as even as a split at view boundaries allows (rank r takes the views
    whose pixel-prefix midpoint falls in [r, r+1) / world of the total)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world size or rank")
    total = float(sum(pixels))
    bounds, acc = [], 0.0
    for p in pixels:
        mid = (acc + 0.5 * p) / total if total > 0 else 0.0
        bounds.append(min(int(mid * world), world - 1))
        acc += p
    start = next((i for i, b in enumerate(bounds) if b >= rank), len(pixels))
    stop = next((i for i, b in enumerate(bounds) if b > rank), len(pixels))
    return start, stop


def flat_gaussians_like(g: Gaussians):
    """Gradient tensors shaped like g's, all views into one flat FP32 buffer."""
    sizes = [getattr(g, k).numel() for k in _FIELDS]
    flat = torch.zeros(sum(sizes), dtype=torch.float32, device=g.means.device)
    parts, off = {}, 0
    for k, s in zip(_FIELDS, sizes):
        parts[k] = flat[off:off + s].view(getattr(g, k).shape)
        off += s
    return flat, Gaussians(sh_degree=g.sh_degree, **parts)


def all_reduce_grads(flat: torch.Tensor, group=None):
    """Sum of every rank's gradient buffer, in place (a no-op without a process group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    return flat


class ShardedStep:
    """One multi-view forward+backward step split across the ranks of `group`.

    cams, dL_list: every view of the step and its dL/dimage ([3,H,W] each); each rank
    keeps its own share.  replay() runs this rank's share (a CUDA graph) and
    all-reduces the gradients, after which `grads` holds the gradient of the whole
    step on every rank."""

    def __init__(self, cams, g: Gaussians, dL_list, group=None, tile=(16, 16), batch=0, device="cuda"):
        import numpy as np
        import torch.distributed as dist
        self.group = group
        dist_on = dist.is_available() and dist.is_initialized()
        self.world = dist.get_world_size(group) if dist_on else 1
        self.rank = dist.get_rank(group) if dist_on else 0
        self.start, self.stop = shard_views([int(c.width) * int(c.height) for c in cams], self.world, self.rank)
        self.cams = list(cams)[self.start:self.stop]
        self.g = g
        self.flat, self.grads = flat_gaussians_like(g)
        self.step = None
        self.rast = None
        if self.cams:
            dL = torch.from_numpy(np.concatenate([np.asarray(d, np.float32).reshape(-1)
                                                  for d in dL_list[self.start:self.stop]])).to(device)
            self.dL = dL
            cfg = H.make_config(tile=tile, batch=batch, persistent=True)
            self.rast = Rasterizer(self.cams, g.n, cfg, device=device)
            self.rast.forward(g)                       # sizes the pair buffers
            self.rast._alloc_pairs(int(self.rast.num_pairs.item() * 1.05) + 4096)
            self.step = GraphStep(self.rast, g, dL, self.grads)

    def replay(self):
        if self.step is not None:
            self.step.replay()
        else:
            self.flat.zero_()                          # no views here: contributes nothing
        all_reduce_grads(self.flat, self.group)

    def status(self) -> int:
        return self.rast.read_status() if self.rast is not None else 0

    def images(self):
        return self.rast.images() if self.rast is not None else []
