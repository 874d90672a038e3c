"""Many cameras per step: one batched launch sequence over all views versus one
launch sequence per view.

BatchedStep: hgs_project over all views, one hgs_bin over global (view, tile)
ids, and persistent compositing kernels that pop (view, tile) items from a
heaviest-first queue; the projection adjoint sums over views.  PerViewStep: the
same path run once per view (n_views = 1, each view with its own persistent tile
queue), the projection adjoint adding into the same gradient buffers
(hgs_config.accumulate).  Both capture their whole
forward+backward step in one CUDA graph, so neither pays per-launch host cost.
"""
from __future__ import annotations

import ctypes

import torch

from . import hgs as H
from .rasterizer import Gaussians, GraphStep, Rasterizer, _vp


def packed_upstream(dL_list, device):
    """Concatenate per-view [3,H,W] arrays into the packed layout of the C ABI."""
    import numpy as np
    flat = np.concatenate([np.asarray(d, np.float32).reshape(-1) for d in dL_list])
    return torch.from_numpy(flat).to(device)


class BatchedStep:
    def __init__(self, cams, g: Gaussians, dL_packed: torch.Tensor, tile=(16, 16), batch=0, device="cuda"):
        self.cfg = H.make_config(tile=tile, batch=batch, persistent=True)
        self.rast = Rasterizer(cams, g.n, self.cfg, device=device)
        self.rast.forward(g)
        self.rast._alloc_pairs(int(self.rast.num_pairs.item() * 1.05) + 4096)
        self.g, self.dL = g, dL_packed
        self.grads = Gaussians.empty_like(g)
        self.step = GraphStep(self.rast, g, dL_packed, self.grads)

    def replay(self):
        self.step.replay()

    def images(self):
        return self.rast.images()

    def status(self):
        return self.rast.read_status()


class PerViewStep:
    def __init__(self, cams, g: Gaussians, dL_list, tile=(16, 16), batch=0, device="cuda"):
        self.g = g
        self.dev = torch.device(device)
        self.rasts = []
        self.dLs = []
        for k, cam in enumerate(cams):
            cfg = H.make_config(tile=tile, batch=batch, persistent=True, accumulate=k > 0)
            r = Rasterizer([cam], g.n, cfg, device=device)
            r.forward(g)
            r._alloc_pairs(int(r.num_pairs.item() * 1.05) + 4096)
            self.rasts.append(r)
            self.dLs.append(torch.from_numpy(dL_list[k].reshape(-1).copy()).to(device))
        self.grads = Gaussians.empty_like(g)
        self.stream = torch.cuda.Stream(self.dev)
        self.graph = torch.cuda.CUDAGraph()
        self.stream.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(self.stream):
            for _ in range(2):
                self._body()
            self.stream.synchronize()
            with torch.cuda.graph(self.graph, stream=self.stream):
                self._body()
        torch.cuda.current_stream(self.dev).wait_stream(self.stream)

    def _body(self):
        for r, dL in zip(self.rasts, self.dLs):
            r.status.zero_()
            r.forward_async(self.g)
            r.rasterize_bwd(dL)
            r.project_bwd(self.g, self.grads)

    def replay(self):
        self.graph.replay()

    def images(self):
        return [r.images()[0] for r in self.rasts]

    def status(self):
        st = 0
        for r in self.rasts:
            st |= r.read_status()
        return st


def time_replays(step, steps, warmup=3):
    """Mean ms per replay, CUDA events around `steps` back-to-back replays."""
    for _ in range(warmup):
        step.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps
