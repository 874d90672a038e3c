"""Fitting half-Gaussians to target images with the differentiable rasterizer.

A usage example and an end-to-end check of the adjoint kernels: the targets are renders
of a hidden synthetic scene, the loss is L1, and the optimiser is Adam with 3D-GS-style
learning rates, except the splitting-plane normals at 0.003, and with the normal and
opacity rates divided by 1.4 every 5000 iterations (supplementary training settings).
There is no dataset, densification or pruning here: it is not a reproduction of the
paper's training.

Parameters are held raw (log-scales, opacity logits) and activated with PyTorch
elementwise ops; the rasterizer takes activated values (hgs_gaussians).

With mip=True the model is Mip-Splatting-HGS: the 3D smoothing filter (mip.py) joins
the activation, with sigma_f from the training cameras, and the rasterizer runs its
2D filter (hgs_config.mip, low-pass 0.1 as in Mip-Splatting).
"""
from __future__ import annotations

import math

import torch

from . import hgs as H
from . import mip as M
from .rasterizer import Gaussians, HGSRasterize, Rasterizer

# base learning rates (3D-GS defaults; normals per the paper)
LR = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "normals": 3e-3, "logit_o1": 5e-2,
      "logit_o2": 5e-2, "sh_dc": 2.5e-3, "sh_rest": 2.5e-3 / 20}
DECAYED = ("normals", "logit_o1", "logit_o2")     # divided by 1.4 every 5000 iterations


class HalfGaussianModel(torch.nn.Module):
    def __init__(self, sc, device="cuda"):
        super().__init__()
        dev = torch.device(device)

        def p(x):
            return torch.nn.Parameter(torch.as_tensor(x, dtype=torch.float32, device=dev).contiguous())

        eps = 1e-6
        self.sh_degree = int(sc.sh_degree)
        self.means = p(sc.means)
        self.log_scales = p(torch.log(torch.as_tensor(sc.scales, dtype=torch.float32)))
        self.quats = p(sc.quats)
        self.normals = p(sc.normals)
        o1 = torch.as_tensor(sc.opac1, dtype=torch.float32).clamp(eps, 1 - eps)
        o2 = torch.as_tensor(sc.opac2, dtype=torch.float32).clamp(eps, 1 - eps)
        self.logit_o1 = p(torch.log(o1 / (1 - o1)))
        self.logit_o2 = p(torch.log(o2 / (1 - o2)))
        sh = torch.as_tensor(sc.sh, dtype=torch.float32).reshape(sc.means.shape[0], -1, 3)
        self.sh_dc = p(sh[:, :1])
        self.sh_rest = p(sh[:, 1:])
        self.register_buffer("filter_sigma", None)      # Mip-Splatting's 3D filter, if set

    def set_3d_filter(self, cams, k=0.2):
        """sigma_f of each kernel from the training cameras (Mip-Splatting recomputes it
        from time to time; it is not differentiated)."""
        self.filter_sigma = M.filter_sigma(self.means, cams, k)

    @property
    def n(self):
        return int(self.means.shape[0])

    def activated(self):
        scales, o1, o2 = torch.exp(self.log_scales), torch.sigmoid(self.logit_o1), torch.sigmoid(self.logit_o2)
        if self.filter_sigma is not None:
            scales, o1, o2 = M.apply_3d_filter(scales, o1, o2, self.filter_sigma)
        return (self.means, scales, self.quats, self.normals, o1, o2,
                torch.cat([self.sh_dc, self.sh_rest], 1).reshape(self.n, -1))

    def render(self, rast: Rasterizer):
        return HGSRasterize.apply(rast, self.sh_degree, *self.activated())

    def param_groups(self, scene_extent=1.0):
        groups = []
        for name in LR:
            lr = LR[name] * (scene_extent if name == "means" else 1.0)
            groups.append({"params": [getattr(self, name)], "lr": lr, "name": name, "base_lr": lr})
        return groups


def decay_lrs(opt, it):
    for g in opt.param_groups:
        if g["name"] in DECAYED:
            g["lr"] = g["base_lr"] / (1.4 ** (it // 5000))


def render_targets(sc, cams, config=None, device="cuda"):
    """Packed target images of a (hidden) scene."""
    r = Rasterizer(cams, sc.n, config or H.make_config(), device=device)
    return r.forward(Gaussians.from_scene(sc, device)).clone()


def fit(init_scene, cams, target, iters=100, config=None, scene_extent=1.0, device="cuda", log_every=0,
        mip=False, filter_every=100):
    """Adam on an L1 loss between the render of `init_scene`'s parameters and `target`
    (packed images of all views).  mip: Mip-Splatting-HGS (3D filter refreshed every
    `filter_every` iterations, 2D filter in the rasterizer).  Returns (model, list of
    per-iteration losses)."""
    model = HalfGaussianModel(init_scene, device)
    if config is None:
        config = H.make_config(mip=True, lowpass=0.1) if mip else H.make_config()
    rast = Rasterizer(cams, model.n, config, device=device)
    opt = torch.optim.Adam(model.param_groups(scene_extent), eps=1e-15)
    losses = []
    for it in range(iters):
        if mip and it % filter_every == 0:
            model.set_3d_filter(cams)
        decay_lrs(opt, it)
        opt.zero_grad(set_to_none=True)
        img = model.render(rast)
        loss = torch.mean(torch.abs(img - target))
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
        if log_every and it % log_every == 0:
            print(f"iter {it}: L1 {losses[-1]:.5f}", flush=True)
        if not math.isfinite(losses[-1]):
            raise FloatingPointError(f"loss is {losses[-1]} at iteration {it}")
    return model, losses
