"""Seeded synthetic inputs for the half-Gaussian rasterizer.

This module only draws random numbers and lays out cameras; it contains none
of the rasterizer's arithmetic (no projection, no SH evaluation, no
compositing).  Both the CUDA path and the FP64 oracle are fed from here, so
that the two sides see bit-identical FP32 inputs.

The workloads stand in for the paper's trained scenes (Mip-NeRF360,
Tanks&Temples, Deep Blending; Sec. 4.1), which are not available.  Their sizes
follow the kernel counts of the rendering-speed ablation table (1.8M-2.9M
kernels, Suppl. C.4) and the opacity shape follows the histogram of Sec. 3.4
(most kernels have one nearly transparent half).

Parameter conventions (what the C-ABI takes):
  means   [N,3]  world position
  scales  [N,3]  linear (already exponentiated) standard deviations
  quats   [N,4]  (w,x,y,z), need not be unit length
  normals [N,3]  splitting-plane normal, need not be unit length
  opac1   [N]    opacity of the half on the side n.(x-mu) >= 0, in [0,1]
  opac2   [N]    opacity of the other half, in [0,1]
  sh      [N,(D+1)^2,3] real SH coefficients, degree D
Cameras: viewmat [3,4] row-major world->camera [R|t], fx, fy, cx, cy, W, H.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Scene", "Camera", "identity_camera", "look_at_camera", "scene_uniform",
    "config1", "config2", "config3", "config4", "config5",
]


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    normals: np.ndarray
    opac1: np.ndarray
    opac2: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.normals[idx].copy(), self.opac1[idx].copy(), self.opac2[idx].copy(),
                     self.sh[idx].copy(), self.sh_degree)

    def arrays(self):
        return (self.means, self.scales, self.quats, self.normals, self.opac1, self.opac2, self.sh)


@dataclasses.dataclass
class Camera:
    viewmat: np.ndarray          # [3,4] float32, world -> camera
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _unit(rng, n, d):
    v = rng.standard_normal((n, d))
    nv = np.linalg.norm(v, axis=1, keepdims=True)
    nv[nv == 0] = 1.0
    return v / nv


def identity_camera(width, height, f, cx=None, cy=None, bg=(0.0, 0.0, 0.0)) -> Camera:
    vm = np.zeros((3, 4), np.float32)
    vm[0, 0] = vm[1, 1] = vm[2, 2] = 1.0
    return Camera(vm, float(f), float(f), float(width / 2 if cx is None else cx),
                  float(height / 2 if cy is None else cy), int(width), int(height), bg=bg)


def look_at_camera(eye, target, up, width, height, f, bg=(0.0, 0.0, 0.0)) -> Camera:
    """Camera at `eye` looking at `target`; camera axes x right, y down, z forward."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    if abs(np.dot(up, fwd)) > 0.999:           # looking along the up axis: swap it
        up = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])          # rows: camera axes in world coordinates
    vm = np.zeros((3, 4), np.float64)
    vm[:, :3] = rot
    vm[:, 3] = -rot @ eye
    return Camera(_f32(vm), float(f), float(f), float(width / 2), float(height / 2),
                  int(width), int(height), bg=bg)


def scene_uniform(rng, n, lo, hi, log_scale_mu, log_scale_sigma, opac_sigma, sh_degree,
                  sh_sigma=0.3, dc_uniform=False) -> Scene:
    means = rng.uniform(lo, hi, size=(n, 3))
    scales = np.exp(rng.normal(log_scale_mu, log_scale_sigma, size=(n, 3)))
    quats = _unit(rng, n, 4)
    normals = _unit(rng, n, 3)
    opac1 = _sigmoid(rng.normal(0.0, opac_sigma, size=n))
    opac2 = _sigmoid(rng.normal(0.0, opac_sigma, size=n))
    nc = (sh_degree + 1) ** 2
    if dc_uniform:
        # DC coefficient drawn on (-sqrt(pi), sqrt(pi)): with the degree-0 basis value
        # 1/(2 sqrt(pi)) and the +0.5 offset the colour is then uniform on [0, 1].
        sh = np.zeros((n, nc, 3))
        sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), size=(n, 3))
    else:
        sh = rng.normal(0.0, sh_sigma, size=(n, nc, 3))
    return Scene(_f32(means), _f32(scales), _f32(quats), _f32(normals), _f32(opac1),
                 _f32(opac2), _f32(sh), sh_degree)


def config1(seed=1):
    """64x64 pinhole (f=64, c=32), identity camera, 1,000 splats, SH degree 0."""
    rng = np.random.default_rng(seed)
    sc = scene_uniform(rng, 1000, [-1, -1, 2], [1, 1, 6], -3.0, 0.5, 1.0, 0, dc_uniform=True)
    return sc, [identity_camera(64, 64, 64.0, 32.0, 32.0)]


def config2(seed=2, n=200_000):
    """1280x720, f=1000, 200k splats in a 10x10x10 box in front of the camera, SH degree 3."""
    rng = np.random.default_rng(seed)
    sc = scene_uniform(rng, n, [-5, -5, 1], [5, 5, 11], -4.0, 0.7, 1.5, 3)
    return sc, [identity_camera(1280, 720, 1000.0, 640.0, 360.0)]


def upstream_grad(seed, cams):
    """dL/dimage ~ N(0,1), one [3,H,W] float32 array per camera."""
    rng = np.random.default_rng(seed)
    return [_f32(rng.standard_normal((3, c.height, c.width))) for c in cams]


def _bimodal_opacity(rng, n):
    lo = math.log(0.05 / 0.95)
    hi = math.log(0.9 / 0.1)
    pick = rng.random(n) < 0.5
    z = np.where(pick, lo, hi) + rng.normal(0.0, 0.25, size=n)
    return _sigmoid(z)


def _blob_means(rng, n, n_blobs=50, blob_sigma=0.5, box=4.0, bg_box=6.0, bg_frac=0.1):
    n_bg = int(round(n * bg_frac))
    n_bl = n - n_bg
    centres = rng.uniform(-box, box, size=(n_blobs, 3))
    which = rng.integers(0, n_blobs, size=n_bl)
    m_bl = centres[which] + rng.normal(0.0, blob_sigma, size=(n_bl, 3))
    m_bg = rng.uniform(-bg_box, bg_box, size=(n_bg, 3))
    means = np.concatenate([m_bl, m_bg], axis=0)
    return means[rng.permutation(n)]


def config3_camera():
    # camera at (0,0,-12) looking along +z: R = I, t = -R*eye = (0,0,12)
    vm = np.zeros((3, 4), np.float32)
    vm[0, 0] = vm[1, 1] = vm[2, 2] = 1.0
    vm[2, 3] = 12.0
    return Camera(vm, 1500.0, 1500.0, 960.0, 540.0, 1920, 1080)


def config3(seed=3, n=3_000_000):
    """Scene-scale step: 3M splats in 50 Gaussian blobs + 10% uniform, 1920x1080, SH degree 3."""
    rng = np.random.default_rng(seed)
    means = _blob_means(rng, n)
    scales = np.exp(rng.normal(-5.0, 1.0, size=(n, 3)))
    quats = _unit(rng, n, 4)
    normals = _unit(rng, n, 3)
    opac1 = _bimodal_opacity(rng, n)
    opac2 = _bimodal_opacity(rng, n)
    sh = rng.normal(0.0, 0.3, size=(n, 16, 3))
    sc = Scene(_f32(means), _f32(scales), _f32(quats), _f32(normals), _f32(opac1), _f32(opac2),
               _f32(sh), 3)
    return sc, [config3_camera()]


RESOLUTIONS = [(640, 360), (1280, 720), (1600, 900), (1920, 1080)]


def fibonacci_cameras(n_views, radius=8.0, seed=104, resolutions=RESOLUTIONS):
    rng = np.random.default_rng(seed)
    cams = []
    golden = math.pi * (3.0 - math.sqrt(5.0))
    for i in range(n_views):
        y = 1.0 - 2.0 * (i + 0.5) / n_views
        rr = math.sqrt(max(0.0, 1.0 - y * y))
        th = golden * i
        eye = radius * np.array([math.cos(th) * rr, y, math.sin(th) * rr])
        w, h = resolutions[int(rng.integers(0, len(resolutions)))]
        f = 0.5 * w / math.tan(math.radians(30.0))
        cams.append(look_at_camera(eye, [0.0, 0.0, 0.0], [0.0, 1.0, 0.0], w, h, f))
    return cams


def config4(seed=4, n=1_000_000, n_views=64):
    """Batched multi-view: 1M splats in [-5,5]^3, 64 cameras on a sphere of radius 8."""
    rng = np.random.default_rng(seed)
    sc = scene_uniform(rng, n, [-5, -5, -5], [5, 5, 5], -4.0, 0.7, 1.5, 3)
    return sc, fibonacci_cameras(n_views)


def config5(n, seed=5, disk_frac=0.3, equal_opacity=False):
    """Stress scene at 1920x1080: config-3 generator plus 30% 100:1 disks whose splitting
    planes are within 5 degrees of containing the ray to the splat centre."""
    sc, cams = config3(seed=seed, n=n)
    rng = np.random.default_rng(seed + 1000)
    cam = cams[0]
    disk = rng.random(n) < disk_frac
    nd = int(disk.sum())
    s = sc.scales[disk].astype(np.float64)
    s[:, 2] = s[:, 0] / 100.0
    s[:, 1] = s[:, 0]
    sc.scales[disk] = _f32(s)
    # camera centre in world coordinates: -R^T t
    rot = cam.viewmat[:, :3].astype(np.float64)
    eye = -rot.T @ cam.viewmat[:, 3].astype(np.float64)
    ray = sc.means[disk].astype(np.float64) - eye
    ray /= np.linalg.norm(ray, axis=1, keepdims=True)
    # a unit vector orthogonal to the ray, then tilt it towards the ray by <= 5 degrees
    tmp = _unit(rng, nd, 3)
    perp = tmp - np.sum(tmp * ray, axis=1, keepdims=True) * ray
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    ang = np.radians(rng.uniform(85.0, 90.0, size=nd))      # angle between n and the ray
    nrm = np.cos(ang)[:, None] * ray + np.sin(ang)[:, None] * perp
    sc.normals[disk] = _f32(nrm)
    if equal_opacity:
        sc.opac2[:] = sc.opac1
    return sc, cams
