"""Mip-Splatting's 3D smoothing filter for half-Gaussians (the Mip-Splatting-HGS variant
of Sec. 4, which swaps Mip-Splatting's kernel for the half-Gaussian one).

The filter caps a kernel's frequency at what the training views can sample.  Each
kernel is convolved in 3D with an isotropic Gaussian of standard deviation
sigma_f = sqrt(k) / nu, where nu is the highest sampling rate (focal length / depth:
pixels per world unit) at which any training camera sees the kernel's centre, and k
(0.2 in Mip-Splatting) sets the filter's width in pixels squared.  The convolution adds
sigma_f^2 I to Sigma^w = R S^2 R^T; I commutes with R, so the result is
R (S^2 + sigma_f^2 I) R^T: scales sqrt(s^2 + sigma_f^2) along the same axes.  As a
normalised convolution it keeps the kernel's mass, which scales the opacity by
sqrt(det Sigma^w / det(Sigma^w + sigma_f^2 I)) = prod_i s_i / sqrt(s_i^2 + sigma_f^2).
For a half-Gaussian both opacities take the factor and the splitting plane is kept:
the filtered kernel is the half-Gaussian of the filtered covariance, as the variant
changes only the kernel inside Mip-Splatting.

This is a transform of the model's parameters (recomputed from the cameras now and
then, not differentiated through nu), applied before the rasterizer; the rasterizer's
part of Mip-Splatting, the 2D filter, is hgs_config.mip.
"""
from __future__ import annotations

import torch


def max_sampling_rate(means: torch.Tensor, cams, margin: float = 1.15) -> torch.Tensor:
    """nu [N]: the largest f / t_z over the cameras whose view frustum (widened by
    `margin`, beyond the near plane) holds the kernel's centre.  Kernels no camera
    sees get the smallest rate among those seen (the widest filter)."""
    means = means.detach()
    nu = torch.zeros(means.shape[0], dtype=means.dtype, device=means.device)
    for cam in cams:
        vm = torch.as_tensor(cam.viewmat, dtype=means.dtype, device=means.device).reshape(3, 4)
        t = means @ vm[:, :3].T + vm[:, 3]
        z = t[:, 2]
        near = float(getattr(cam, "near", 0.2))
        safe = torch.where(z > near, z, torch.ones_like(z))
        ok = (z > near) & ((t[:, 0] / safe).abs() <= margin * 0.5 * cam.width / cam.fx) & \
             ((t[:, 1] / safe).abs() <= margin * 0.5 * cam.height / cam.fy)
        rate = torch.where(ok, float(max(cam.fx, cam.fy)) / safe, torch.zeros_like(z))
        nu = torch.maximum(nu, rate)
    seen = nu > 0
    if bool(seen.any()):
        nu = torch.where(seen, nu, nu[seen].min())
    else:
        nu = torch.ones_like(nu)
    return nu


def filter_sigma(means: torch.Tensor, cams, k: float = 0.2, margin: float = 1.15) -> torch.Tensor:
    """sigma_f [N] = sqrt(k) / nu."""
    return (k ** 0.5) / max_sampling_rate(means, cams, margin)


def apply_3d_filter(scales: torch.Tensor, opac1: torch.Tensor, opac2: torch.Tensor, sigma_f: torch.Tensor):
    """Scales, opacity1, opacity2 of the filtered kernels (differentiable in the
    parameters; sigma_f is held fixed)."""
    s2 = scales * scales
    var = (sigma_f * sigma_f).unsqueeze(-1)
    eff = torch.sqrt(s2 + var)
    factor = torch.prod(scales / eff, dim=-1)
    return eff, opac1 * factor, opac2 * factor
