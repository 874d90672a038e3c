"""Rasterizer: buffers, capacity handling, CUDA-graph capture and autograd around
the C ABI.  PyTorch only provides device memory, streams and autograd; every
step of the path runs in libhgs's kernels (via paper_2406_02720_b300.hgs).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import hgs as H

_FIELDS = ("means", "scales", "quats", "normals", "opac1", "opac2", "sh")


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


@dataclass
class Gaussians:
    """Half-Gaussian parameters as contiguous FP32 CUDA tensors (layout of hgs_gaussians)."""
    means: torch.Tensor
    scales: torch.Tensor
    quats: torch.Tensor
    normals: torch.Tensor
    opac1: torch.Tensor
    opac2: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_scene(sc, device="cuda") -> "Gaussians":
        t = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k), dtype=np.float32)).to(device)
             for k in _FIELDS}
        return Gaussians(sh_degree=int(sc.sh_degree), **t)

    @staticmethod
    def empty_like(g: "Gaussians") -> "Gaussians":
        return Gaussians(sh_degree=g.sh_degree, **{k: torch.empty_like(getattr(g, k)) for k in _FIELDS})

    def tensors(self):
        return [getattr(self, k) for k in _FIELDS]

    def c_struct(self) -> H.HgsGaussians:
        s = H.HgsGaussians()
        for k in _FIELDS:
            setattr(s, k, _vp(getattr(self, k)))
        s.n = self.n
        s.sh_degree = self.sh_degree
        return s

    def c_grads(self) -> H.HgsGaussianGrads:
        s = H.HgsGaussianGrads()
        for k in _FIELDS:
            setattr(s, k, _vp(getattr(self, k)))
        return s


class Rasterizer:
    """Owns every buffer of the path for a fixed set of camera sizes and splat count.

    forward(g)      -> image [3*total_pixels] (views packed, [3,H,W] each)
    backward(g, dL) -> Gaussians of gradients
    Pair capacity grows automatically when a step reports HGS_DEV_CAPACITY (the
    step is then re-run outside any graph)."""

    def __init__(self, cams, n, config=None, pair_capacity=None, device="cuda", keep_keys=False):
        self.device = torch.device(device)
        self.keep_keys = keep_keys          # also write the sorted 64-bit keys (not needed to render)
        self.cfg = config if config is not None else H.make_config()
        self.cams_list = list(cams)
        self.n_views = len(self.cams_list)
        self.n = int(n)
        self.cams_host = H.make_cameras(self.cams_list)
        raw = bytes(ctypes.string_at(ctypes.addressof(self.cams_host), ctypes.sizeof(self.cams_host)))
        self.cams_dev = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(self.device)
        self.total_tiles, self.total_pixels = H.hgs_layout(self.cams_host, self.n_views, self.cfg)
        vn = self.n * self.n_views
        f32, i32, dev = torch.float32, torch.int32, self.device
        self.rec = torch.empty((vn, 16), dtype=f32, device=dev)
        self.depth = torch.empty(vn, dtype=f32, device=dev)
        self.rect = torch.empty((vn, 4), dtype=i32, device=dev)
        self.tiles = torch.empty(vn, dtype=i32, device=dev)
        self.fp64_list = torch.empty(vn + 1, dtype=i32, device=dev)
        self.status = torch.zeros(1, dtype=i32, device=dev)
        self.num_pairs = torch.zeros(1, dtype=torch.int64, device=dev)
        self.ranges = torch.empty((self.total_tiles, 2), dtype=i32, device=dev)
        self.image = torch.empty(3 * self.total_pixels, dtype=f32, device=dev)
        self.final_T = torch.empty(self.total_pixels, dtype=f32, device=dev)
        self.n_contrib = torch.empty(self.total_pixels, dtype=i32, device=dev)
        self.grad2d = torch.empty((vn, 12), dtype=f32, device=dev)
        self._from_forward = False      # the last call on grad2d / render_ws was render_fwd
        rws = H.hgs_render_workspace_size(self.cams_host, self.n_views, self.cfg, self.n)
        self.render_ws = torch.empty(max(rws, 16), dtype=torch.uint8, device=dev)
        self.capacity = 0
        self._alloc_pairs(pair_capacity if pair_capacity else max(4096, 4 * vn))

    # -- buffers ------------------------------------------------------------------------
    def _alloc_pairs(self, cap):
        cap = int(min(max(cap, 1), H.HGS_MAX_PAIRS))
        if cap == self.capacity:
            return
        self.capacity = cap
        self.keys = torch.empty(cap if self.keep_keys else 0, dtype=torch.int64, device=self.device)
        self.ids = torch.empty(cap, dtype=torch.int32, device=self.device)
        wsb = H.hgs_bin_workspace_size(self.n, self.n_views, cap)
        self.bin_ws = torch.empty(wsb, dtype=torch.uint8, device=self.device)
        # visibility mask: written by the forward compositing, read by the backward
        self.vis = torch.empty(H.hgs_vis_words(self.cams_host, self.n_views, self.cfg, cap), dtype=torch.int32,
                               device=self.device)

    def proj_struct(self) -> H.HgsProj:
        p = H.HgsProj()
        p.rec, p.depth, p.rect, p.tiles = _vp(self.rec), _vp(self.depth), _vp(self.rect), _vp(self.tiles)
        p.fp64_list = _vp(self.fp64_list)
        return p

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    # -- the four steps ------------------------------------------------------------------
    def project(self, g: Gaussians):
        H.hgs_project(g.c_struct(), self.cams_host, _vp(self.cams_dev), self.n_views, self.cfg,
                      self.proj_struct(), _vp(self.status), self._stream())

    def bin(self):
        H.hgs_bin(self.proj_struct(), self.n, self.cams_host, self.n_views, self.cfg, _vp(self.bin_ws),
                  self.bin_ws.numel(), self.capacity, _vp(self.keys), _vp(self.ids), _vp(self.ranges),
                  _vp(self.num_pairs), _vp(self.status), self._stream())

    def render_fwd(self, image: torch.Tensor = None):
        """Composites into self.image, or into `image` (same size and dtype) when given,
        e.g. a staging buffer that a copy to the host reads next."""
        if image is None:
            image = self.image
        elif (image.numel() != self.image.numel() or image.dtype != self.image.dtype
              or image.device != self.image.device or not image.is_contiguous()):
            raise ValueError("image buffer must match the rasterizer's image (size, dtype, device, contiguous)")
        # the kernel also clears grad2d for the backward that follows it on the stream
        H.hgs_render_fwd(self.proj_struct(), self.n, _vp(self.ids), _vp(self.ranges), self.cams_host,
                         _vp(self.cams_dev), self.n_views, self.cfg, _vp(self.render_ws), self.render_ws.numel(),
                         _vp(image), _vp(self.final_T), _vp(self.n_contrib), _vp(self.vis), self.vis.numel(),
                         _vp(self.grad2d), _vp(self.status), self._stream())
        self._from_forward = True

    def rasterize_bwd(self, dL_dimage: torch.Tensor):
        # right after render_fwd, grad2d is already zero and the tile queue in render_ws is
        # built; a second backward after one forward clears and builds them again
        after_fwd, self._from_forward = self._from_forward, False
        H.hgs_rasterize_bwd(self.proj_struct(), self.n, _vp(self.ids), _vp(self.ranges), self.cams_host,
                            _vp(self.cams_dev), self.n_views, self.cfg, _vp(self.render_ws),
                            self.render_ws.numel(), _vp(self.final_T), _vp(self.n_contrib), _vp(self.vis),
                            self.vis.numel(), _vp(dL_dimage), _vp(self.grad2d), after_fwd, _vp(self.status),
                            self._stream())

    def project_bwd(self, g: Gaussians, out: Gaussians):
        H.hgs_project_bwd(g.c_struct(), self.cams_host, _vp(self.cams_dev), self.n_views, self.cfg,
                          _vp(self.grad2d), out.c_grads(), _vp(self.fp64_list), _vp(self.status), self._stream())

    # -- composite steps ---------------------------------------------------------------
    def forward_async(self, g: Gaussians):
        self.project(g)
        self.bin()
        self.render_fwd()
        return self.image

    def backward_async(self, g: Gaussians, dL_dimage: torch.Tensor, out: Gaussians):
        self.rasterize_bwd(dL_dimage)
        self.project_bwd(g, out)
        return out

    def stats(self, dL_dimage: torch.Tensor) -> dict:
        """Work counters of one forward + backward compositing pass (hgs_render_stats)."""
        cnt = torch.zeros(8, dtype=torch.int64, device=self.device)
        self._from_forward = False           # its own forward and backward reuse grad2d and render_ws
        H.hgs_render_stats(self.proj_struct(), self.n, _vp(self.ids), _vp(self.ranges), self.cams_host,
                           _vp(self.cams_dev), self.n_views, self.cfg, _vp(self.render_ws), self.render_ws.numel(),
                           _vp(self.image), _vp(self.final_T), _vp(self.n_contrib), _vp(self.vis), self.vis.numel(),
                           _vp(dL_dimage), _vp(self.grad2d), _vp(cnt), _vp(self.status), self._stream())
        self._raise_status(self.read_status())
        v = cnt.cpu().tolist()
        return {k: int(v[i]) for i, k in enumerate(H.STAT_NAMES)}

    def read_status(self) -> int:
        torch.cuda.current_stream(self.device).synchronize()
        return int(self.status.item())

    def clear_status(self):
        self.status.zero_()

    def forward(self, g: Gaussians) -> torch.Tensor:
        """Projection, binning and compositing; grows the pair capacity and re-runs if needed."""
        assert g.n == self.n
        for _ in range(4):
            self.clear_status()
            self.project(g)
            self.bin()
            st = self.read_status()
            if st & H.HGS_DEV_CAPACITY:
                self._alloc_pairs(int(self.num_pairs.item() * 1.25) + 1024)
                continue
            self._raise_status(st)
            self.render_fwd()
            self._raise_status(self.read_status())
            return self.image
        raise H.HgsError("pair capacity could not be satisfied")

    def backward(self, g: Gaussians, dL_dimage: torch.Tensor, out: Gaussians = None) -> Gaussians:
        out = out if out is not None else Gaussians.empty_like(g)
        self.backward_async(g, dL_dimage.contiguous(), out)
        self._raise_status(self.read_status())
        return out

    @staticmethod
    def _raise_status(st):
        if st:
            names = [n for b, n in ((1, "capacity"), (2, "timeout"), (4, "bounds")) if st & b]
            raise H.HgsError("device status: " + ", ".join(names))

    # -- views of the packed outputs ---------------------------------------------------------
    def view_slices(self):
        out, off = [], 0
        for c in self.cams_list:
            out.append((off, int(c.width), int(c.height)))
            off += int(c.width) * int(c.height)
        return out

    def images(self, flat=None):
        flat = self.image if flat is None else flat
        return [flat[3 * o:3 * (o + w * h)].view(3, h, w) for o, w, h in self.view_slices()]

    def per_pixel(self, flat):
        return [flat[o:o + w * h].view(h, w) for o, w, h in self.view_slices()]

    def sorted_pairs(self):
        k = int(self.num_pairs.item())
        return (self.keys[:k] if self.keep_keys else None), self.ids[:k]


class HGSRasterize(torch.autograd.Function):
    """image = render(params); backward calls the hand-written adjoint kernels."""

    @staticmethod
    def forward(ctx, rast: Rasterizer, sh_degree: int, means, scales, quats, normals, opac1, opac2, sh):
        g = Gaussians(means.contiguous(), scales.contiguous(), quats.contiguous(), normals.contiguous(),
                      opac1.contiguous(), opac2.contiguous(), sh.contiguous(), sh_degree)
        img = rast.forward(g).clone()
        ctx.rast = rast
        ctx.g = g
        return img

    @staticmethod
    def backward(ctx, dimage):
        out = ctx.rast.backward(ctx.g, dimage.contiguous())
        return (None, None, *out.tensors())


def render(rast: Rasterizer, g: Gaussians, requires_grad=True):
    """Differentiable render of all views (packed image)."""
    return HGSRasterize.apply(rast, g.sh_degree, *g.tensors())


class GraphStep:
    """A whole forward+backward step (project, bin, composite, adjoint) captured once
    in a CUDA graph and replayed.  Inputs are read from `g` and `dL`, outputs land in
    rast.image / grads; the pair capacity must already fit (run rast.forward once)."""

    def __init__(self, rast: Rasterizer, g: Gaussians, dL: torch.Tensor, grads: Gaussians, backward=True):
        self.rast, self.g, self.dL, self.grads = rast, g, dL, grads
        self.stream = torch.cuda.Stream(rast.device)
        self.graph = torch.cuda.CUDAGraph()
        self.stream.wait_stream(torch.cuda.current_stream(rast.device))
        with torch.cuda.stream(self.stream):
            for _ in range(2):                  # warm the stream (lazy init) before capture
                self._body(backward)
            self.stream.synchronize()
            with torch.cuda.graph(self.graph, stream=self.stream):
                self._body(backward)
        torch.cuda.current_stream(rast.device).wait_stream(self.stream)

    def _body(self, backward):
        self.rast.status.zero_()
        self.rast.forward_async(self.g)
        if backward:
            self.rast.backward_async(self.g, self.dL, self.grads)

    def replay(self):
        self.graph.replay()
