"""ctypes binding of the C ABI in include/hgs.h (libhgs.so).

Argument marshalling only: every function here forwards to the entry point of
the same name, passing device pointers and the CUDA stream; the rasterizer's
arithmetic runs in the library's kernels.  If the library is missing it is
built with nvcc; if that fails, importing raises (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, c_float, c_int, c_int64, c_size_t, c_uint32, c_uint64, c_void_p

from . import build as _build

HGS_OK, HGS_ERR_INVALID, HGS_ERR_CAPACITY, HGS_ERR_CUDA, HGS_ERR_TIMEOUT, HGS_ERR_UNSUPPORTED = range(6)
HGS_DEV_CAPACITY, HGS_DEV_TIMEOUT, HGS_DEV_BOUNDS = 1, 2, 4
HGS_MAX_VIEWS = 256
HGS_MAX_PAIRS = (1 << 30) - 1
HEADER = os.path.join(_build.INCLUDE, "hgs.h")


class HgsCamera(ctypes.Structure):
    _fields_ = [("viewmat", c_float * 12), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("width", c_int), ("height", c_int), ("near_plane", c_float),
                ("bg", c_float * 3)]


class HgsConfig(ctypes.Structure):
    _fields_ = [("tile_w", c_int), ("tile_h", c_int), ("batch", c_int), ("lowpass", c_float),
                ("fov_clamp", c_int), ("plain", c_int), ("persistent", c_int), ("accumulate", c_int),
                ("rect_mode", c_int), ("mip", c_int)]


class HgsGaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p), ("normals", c_void_p),
                ("opac1", c_void_p), ("opac2", c_void_p), ("sh", c_void_p), ("n", c_int),
                ("sh_degree", c_int)]


class HgsGaussianGrads(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p), ("normals", c_void_p),
                ("opac1", c_void_p), ("opac2", c_void_p), ("sh", c_void_p)]


class HgsProj(ctypes.Structure):
    _fields_ = [("rec", c_void_p), ("depth", c_void_p), ("rect", c_void_p), ("tiles", c_void_p),
                ("fp64_list", c_void_p)]


class HgsError(RuntimeError):
    pass


_LIB = None
_CAM_P = POINTER(HgsCamera)
_CFG_P = POINTER(HgsConfig)


def lib_path() -> str:
    return _build.LIB


def lib():
    """Loads libhgs.so (building it first if it is missing or older than its sources)."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp = c_void_p
        L.hgs_version.restype = c_int
        L.hgs_status_string.restype = ctypes.c_char_p
        L.hgs_status_string.argtypes = [c_int]
        L.hgs_layout.restype = c_int
        L.hgs_layout.argtypes = [_CAM_P, c_int, _CFG_P, POINTER(c_int), POINTER(c_int64)]
        L.hgs_bin_workspace_size.restype = c_size_t
        L.hgs_bin_workspace_size.argtypes = [c_int, c_int, c_size_t]
        L.hgs_render_workspace_size.restype = c_size_t
        L.hgs_render_workspace_size.argtypes = [_CAM_P, c_int, _CFG_P, c_int]
        L.hgs_vis_words.restype = c_size_t
        L.hgs_vis_words.argtypes = [_CAM_P, c_int, _CFG_P, c_size_t]
        L.hgs_project.restype = c_int
        L.hgs_project.argtypes = [POINTER(HgsGaussians), _CAM_P, vp, c_int, _CFG_P, POINTER(HgsProj), vp, vp]
        L.hgs_bin.restype = c_int
        L.hgs_bin.argtypes = [POINTER(HgsProj), c_int, _CAM_P, c_int, _CFG_P, vp, c_size_t, c_size_t,
                              vp, vp, vp, vp, vp, vp]
        L.hgs_bin_static.restype = c_int
        L.hgs_bin_static.argtypes = [POINTER(HgsProj), c_int, _CAM_P, c_int, _CFG_P, c_size_t, vp, vp, vp, vp, vp,
                                     vp]
        L.hgs_render_fwd.restype = c_int
        L.hgs_render_fwd.argtypes = [POINTER(HgsProj), c_int, vp, vp, _CAM_P, vp, c_int, _CFG_P, vp,
                                     c_size_t, vp, vp, vp, vp, c_size_t, vp, vp, vp]
        L.hgs_rasterize_bwd.restype = c_int
        L.hgs_rasterize_bwd.argtypes = [POINTER(HgsProj), c_int, vp, vp, _CAM_P, vp, c_int, _CFG_P, vp,
                                        c_size_t, vp, vp, vp, c_size_t, vp, vp, c_int, vp, vp]
        L.hgs_project_bwd.restype = c_int
        L.hgs_project_bwd.argtypes = [POINTER(HgsGaussians), _CAM_P, vp, c_int, _CFG_P, vp,
                                      POINTER(HgsGaussianGrads), vp, vp, vp]
        L.hgs_render_stats.restype = c_int
        L.hgs_render_stats.argtypes = [POINTER(HgsProj), c_int, vp, vp, _CAM_P, vp, c_int, _CFG_P, vp, c_size_t,
                                       vp, vp, vp, vp, c_size_t, vp, vp, vp, vp, vp]
        L.hgs_render_bwd.restype = c_int
        L.hgs_render_bwd.argtypes = [POINTER(HgsGaussians), POINTER(HgsProj), vp, vp, _CAM_P, vp, c_int,
                                     _CFG_P, vp, c_size_t, vp, vp, vp, c_size_t, vp, vp,
                                     POINTER(HgsGaussianGrads), vp, vp]
        L.hgs_probe_peak.restype = c_int
        L.hgs_probe_peak.argtypes = [c_int, c_int, c_int, vp, POINTER(ctypes.c_double), vp]
        L.hgs_selftest_wait.restype = c_int
        L.hgs_selftest_wait.argtypes = [vp, vp]
        _LIB = L
    return _LIB


def declared_functions():
    """Names of the functions include/hgs.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hgs_[a-z_0-9]+)\s*\(", txt)))


def _check(st: int, what: str):
    if st != HGS_OK:
        msg = lib().hgs_status_string(st).decode()
        raise HgsError(f"{what}: {msg} ({st})")


# ---- entry points (same names as the C ABI) --------------------------------------------
def hgs_version() -> int:
    return int(lib().hgs_version())


def hgs_status_string(st: int) -> str:
    return lib().hgs_status_string(st).decode()


def hgs_layout(cams_host, n_views, cfg):
    tiles = c_int(0)
    pix = c_int64(0)
    _check(lib().hgs_layout(cams_host, n_views, ctypes.byref(cfg), ctypes.byref(tiles), ctypes.byref(pix)),
           "hgs_layout")
    return tiles.value, pix.value


def hgs_bin_workspace_size(n, n_views, pair_capacity) -> int:
    return int(lib().hgs_bin_workspace_size(n, n_views, pair_capacity))


def hgs_render_workspace_size(cams_host, n_views, cfg, n) -> int:
    return int(lib().hgs_render_workspace_size(cams_host, n_views, ctypes.byref(cfg), n))


def hgs_vis_words(cams_host, n_views, cfg, pair_capacity) -> int:
    return int(lib().hgs_vis_words(cams_host, n_views, ctypes.byref(cfg), pair_capacity))


def hgs_project(g, cams_host, cams_dev, n_views, cfg, out, dev_status, stream):
    _check(lib().hgs_project(ctypes.byref(g), cams_host, cams_dev, n_views, ctypes.byref(cfg),
                             ctypes.byref(out), dev_status, stream), "hgs_project")


def hgs_bin(proj, n, cams_host, n_views, cfg, ws, ws_bytes, pair_capacity, keys_out, ids_out, ranges,
            dev_num_pairs, dev_status, stream):
    _check(lib().hgs_bin(ctypes.byref(proj), n, cams_host, n_views, ctypes.byref(cfg), ws, ws_bytes,
                         pair_capacity, keys_out, ids_out, ranges, dev_num_pairs, dev_status, stream), "hgs_bin")


HGS_BIN_STATIC_SCRATCH_BYTES = 32 << 20


def hgs_bin_static(proj, n, cams_host, n_views, cfg, pair_capacity, keys_out, ids_out, ranges, dev_num_pairs,
                   dev_status, stream):
    """hgs_bin with the scratch workspace in the library's fixed device array (no
    allocation by the caller or the call)."""
    _check(lib().hgs_bin_static(ctypes.byref(proj), n, cams_host, n_views, ctypes.byref(cfg), pair_capacity,
                                keys_out, ids_out, ranges, dev_num_pairs, dev_status, stream), "hgs_bin_static")


def hgs_render_fwd(proj, n, ids, ranges, cams_host, cams_dev, n_views, cfg, ws, ws_bytes, image, final_T,
                   n_contrib, vis, vis_words, grad2d_clear, dev_status, stream):
    _check(lib().hgs_render_fwd(ctypes.byref(proj), n, ids, ranges, cams_host, cams_dev, n_views,
                                ctypes.byref(cfg), ws, ws_bytes, image, final_T, n_contrib, vis, vis_words,
                                grad2d_clear, dev_status, stream), "hgs_render_fwd")


def hgs_rasterize_bwd(proj, n, ids, ranges, cams_host, cams_dev, n_views, cfg, ws, ws_bytes, final_T,
                      n_contrib, vis, vis_words, dL_dimage, grad2d, from_forward, dev_status, stream):
    _check(lib().hgs_rasterize_bwd(ctypes.byref(proj), n, ids, ranges, cams_host, cams_dev, n_views,
                                   ctypes.byref(cfg), ws, ws_bytes, final_T, n_contrib, vis, vis_words, dL_dimage,
                                   grad2d, int(from_forward), dev_status, stream), "hgs_rasterize_bwd")


def hgs_project_bwd(g, cams_host, cams_dev, n_views, cfg, grad2d, out, fp64_list, dev_status, stream):
    _check(lib().hgs_project_bwd(ctypes.byref(g), cams_host, cams_dev, n_views, ctypes.byref(cfg), grad2d,
                                 ctypes.byref(out), fp64_list, dev_status, stream), "hgs_project_bwd")


def hgs_render_bwd(g, proj, ids, ranges, cams_host, cams_dev, n_views, cfg, ws, ws_bytes, final_T, n_contrib,
                   vis, vis_words, dL_dimage, grad2d, out, dev_status, stream):
    _check(lib().hgs_render_bwd(ctypes.byref(g), ctypes.byref(proj), ids, ranges, cams_host, cams_dev, n_views,
                                ctypes.byref(cfg), ws, ws_bytes, final_T, n_contrib, vis, vis_words, dL_dimage,
                                grad2d, ctypes.byref(out), dev_status, stream), "hgs_render_bwd")


def hgs_render_stats(proj, n, ids, ranges, cams_host, cams_dev, n_views, cfg, ws, ws_bytes, image, final_T,
                     n_contrib, vis, vis_words, dL_dimage, grad2d, counters, dev_status, stream):
    _check(lib().hgs_render_stats(ctypes.byref(proj), n, ids, ranges, cams_host, cams_dev, n_views,
                                  ctypes.byref(cfg), ws, ws_bytes, image, final_T, n_contrib, vis, vis_words,
                                  dL_dimage, grad2d, counters, dev_status, stream), "hgs_render_stats")


def hgs_probe_peak(kind, blocks_per_sm, iters, sink, stream) -> float:
    """Enqueues the FMA (kind 0) or ex2 (kind 1) issue-rate probe; returns the
    lane-operations it performs."""
    ops = ctypes.c_double(0.0)
    _check(lib().hgs_probe_peak(kind, blocks_per_sm, iters, sink, ctypes.byref(ops), stream), "hgs_probe_peak")
    return ops.value


def hgs_selftest_wait(dev_status, stream):
    """Enqueues a wait that nothing ends: it runs out at its bound and sets
    HGS_DEV_TIMEOUT in *dev_status."""
    _check(lib().hgs_selftest_wait(dev_status, stream), "hgs_selftest_wait")


STAT_NAMES = ["fwd_visit", "fwd_full", "fwd_comp", "bwd_visit", "bwd_full", "bwd_contrib", "bwd_warp_red",
              "bwd_atomic"]


# ---- struct builders ----------------------------------------------------------------------
def make_config(tile=(16, 16), batch=0, lowpass=0.3, fov_clamp=True, plain=False, persistent=True,
                accumulate=False, rect_mode=0, mip=False) -> HgsConfig:
    """hgs_config with this package's defaults: 16x16 tiles, per-direction batch,
    3D-GS low-pass and FOV clamp, half-Gaussian weights, and compositing as persistent
    blocks over the heaviest-first tile queue (faster than one block per tile even for
    a single view: 3.26 vs 3.32 ms per fwd+bwd step at 3M splats, 1080p)."""
    c = HgsConfig()
    c.tile_w, c.tile_h = int(tile[0]), int(tile[1])
    c.batch = int(batch)
    c.lowpass = float(lowpass)
    c.fov_clamp = 1 if fov_clamp else 0
    c.plain = 1 if plain else 0
    c.persistent = 1 if persistent else 0
    c.accumulate = 1 if accumulate else 0
    c.rect_mode = int(rect_mode)
    c.mip = 1 if mip else 0
    return c


def make_cameras(cams):
    """Host array of HgsCamera from objects with viewmat/fx/fy/cx/cy/width/height/near/bg."""
    arr = (HgsCamera * len(cams))()
    for i, cam in enumerate(cams):
        vm = [float(x) for x in __import__("numpy").asarray(cam.viewmat, dtype="float32").reshape(12)]
        for k in range(12):
            arr[i].viewmat[k] = vm[k]
        arr[i].fx, arr[i].fy = float(cam.fx), float(cam.fy)
        arr[i].cx, arr[i].cy = float(cam.cx), float(cam.cy)
        arr[i].width, arr[i].height = int(cam.width), int(cam.height)
        arr[i].near_plane = float(getattr(cam, "near", 0.2))
        bg = getattr(cam, "bg", (0.0, 0.0, 0.0))
        for k in range(3):
            arr[i].bg[k] = float(bg[k])
    return arr
