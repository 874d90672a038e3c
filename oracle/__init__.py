"""FP64 CPU oracle for the 3D half-Gaussian splatting rasterizer.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the bench's
CPU-baseline leg call it; the product path never does.  It shares no code
with the CUDA path (hgs_oracle.c is plain C, compiled by oracle/build.py).

Each function cites the part of the paper it follows; see hgs_oracle.c for the
step-by-step arithmetic.  Scenes and cameras are duck-typed: any object with
the attributes of the generator's Scene / Camera works.

Every function here is pinned by a `-m "not gpu"` test in tests/test_oracle_*.py
(quadrature along the ray, closed-form single splats, the alpha1 = alpha2
reduction, complement symmetry, SH against scipy, brute-force binning, and
central finite differences for the adjoint).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int, c_long, c_uint32, c_uint64, c_ubyte

import numpy as np

from . import build as _build

CULLED, NORMAL, STEP, HALF = 0, 1, 2, 3
G2D_FIELDS = ["mu_x", "mu_y", "conic_a", "conic_b", "conic_c", "wp_x", "wp_y",
              "alpha1", "alpha2", "r", "g", "b"]


class OrCamera(ctypes.Structure):
    _fields_ = [("viewmat", c_double * 12), ("fx", c_double), ("fy", c_double),
                ("cx", c_double), ("cy", c_double), ("width", c_int), ("height", c_int),
                ("near_plane", c_double), ("bg", c_double * 3)]


class OrOpts(ctypes.Structure):
    _fields_ = [("tile_w", c_int), ("tile_h", c_int), ("sh_degree", c_int),
                ("fov_clamp", c_int), ("plain", c_int), ("rect_mode", c_int), ("mip", c_int),
                ("lowpass", c_double)]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp, fp, ip = POINTER(c_double), POINTER(c_float), POINTER(c_int)
        L.or_abi_version.restype = c_int
        L.or_num_threads.restype = c_int
        L.or_set_num_threads.argtypes = [c_int]
        L.or_project.argtypes = [c_int, dp, dp, dp, dp, dp, dp, dp, POINTER(OrCamera), POINTER(OrOpts),
                                 ip, fp, fp, ip, ip, fp, fp, dp, dp, dp, dp, dp, dp]
        L.or_bin.argtypes = [c_int, ip, ip, fp, c_int, c_int, POINTER(c_ubyte), c_long,
                             POINTER(c_uint64), POINTER(c_uint32), POINTER(c_uint32),
                             POINTER(c_long)]
        L.or_bin.restype = c_long
        L.or_render_fwd.argtypes = [c_int, ip, dp, dp, dp, dp, dp, dp, POINTER(c_uint32),
                                    POINTER(c_uint32), POINTER(OrCamera), POINTER(OrOpts),
                                    POINTER(c_ubyte), dp, dp, ip, dp, dp, dp, ip,
                                    dp, dp, dp, dp, POINTER(c_ubyte), POINTER(c_ubyte)]
        L.or_error_basis.argtypes = [c_int, dp, dp, dp, dp, POINTER(OrCamera), POINTER(OrOpts), ip,
                                     POINTER(c_ubyte), dp, dp]
        L.or_pair_bands.argtypes = [c_int, ip, dp, dp, dp, dp, dp, dp, c_int, c_int, c_int, ip, dp, dp, dp, dp]
        L.or_render_bwd.argtypes = [c_int, ip, dp, dp, dp, dp, dp, dp, POINTER(c_uint32),
                                    POINTER(c_uint32), POINTER(OrCamera), POINTER(OrOpts),
                                    POINTER(c_ubyte), dp, dp, dp, dp]
        L.or_project_bwd.argtypes = [c_int, dp, dp, dp, dp, dp, dp, dp, POINTER(OrCamera),
                                     POINTER(OrOpts), ip, dp, dp, dp, dp, dp, dp, dp, dp]
        L.or_eval_splat.argtypes = [dp, dp, dp, dp, POINTER(OrCamera), POINTER(OrOpts), c_int,
                                    dp, dp, dp, dp]
        L.or_eval_splat.restype = c_int
        L.or_sh_eval.argtypes = [c_int, c_int, dp, dp]
        L.or_alg1_flat_cov.argtypes = [dp, dp, dp]
        _LIB = L
    return _LIB


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(k: int) -> None:
    """Threads of the oracle's OpenMP loops from now on (k >= 1)."""
    lib().or_set_num_threads(int(k))


def _p(a, ct):
    return a.ctypes.data_as(POINTER(ct))


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_camera(cam) -> OrCamera:
    c = OrCamera()
    vm = np.asarray(cam.viewmat, np.float64).reshape(12)
    for i in range(12):
        c.viewmat[i] = float(vm[i])
    # the camera of the C ABI is binary32 (hgs_camera): take the same binary32 values
    # for the intrinsics, the near plane and the background as for the view matrix
    f32 = lambda x: float(np.float32(x))      # noqa: E731
    c.fx, c.fy, c.cx, c.cy = f32(cam.fx), f32(cam.fy), f32(cam.cx), f32(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_plane = f32(getattr(cam, "near", 0.2))
    bg = getattr(cam, "bg", (0.0, 0.0, 0.0))
    for i in range(3):
        c.bg[i] = f32(bg[i])
    return c


def make_opts(tile=(16, 16), sh_degree=0, lowpass=0.3, plain=False, fov_clamp=True, rect_mode=0,
              mip=False) -> OrOpts:
    o = OrOpts()
    o.rect_mode = int(rect_mode)
    o.mip = 1 if mip else 0
    o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
    o.sh_degree = int(sh_degree)
    o.fov_clamp = 1 if fov_clamp else 0
    o.plain = 1 if plain else 0
    # the GPU receives the low-pass as binary32; use the same value here
    o.lowpass = float(np.float32(lowpass))
    return o


def _scene64(sc):
    return dict(means=_d(sc.means).reshape(-1, 3), scales=_d(sc.scales).reshape(-1, 3),
                quats=_d(sc.quats).reshape(-1, 4), normals=_d(sc.normals).reshape(-1, 3),
                opac1=_d(sc.opac1).reshape(-1), opac2=_d(sc.opac2).reshape(-1),
                sh=_d(sc.sh).reshape(sc.means.shape[0], -1, 3))


def grid(cam, tile):
    tx = (int(cam.width) + tile[0] - 1) // tile[0]
    ty = (int(cam.height) + tile[1] - 1) // tile[1]
    return tx, ty


def project(sc, cam, tile=(16, 16), lowpass=0.3, fov_clamp=True, rect_mode=0, mip=False, errmat=True,
            err_sel=None):
    """Per-splat projection (Eq. 2-5, 7-8; SH colour), plus canonical binning fields.
    rect_mode 0: the 3-sigma square of 3D-GS; 1: per-half 3-sigma extents (Sec. 3.4);
    2: the same with the splitting edge from Algorithm 1's flattened covariance.
    mip: the low-pass as Mip-Splatting's mass-preserving 2D filter; "opac1"/"opac2" are
    then the compensated opacities the compositing uses ("comp" holds the factor).
    errmat: also the FP32 error model's per-splat matrix "errmat" [N,15] (see
    error_basis), for the splats selected by err_sel [N] bool (all if None)."""
    s = _scene64(sc)
    n = s["means"].shape[0]
    o = make_opts(tile, sc.sh_degree, lowpass, False, fov_clamp, rect_mode, mip)
    c = make_camera(cam)
    out = dict(mode=np.zeros(n, np.int32), depth=np.zeros(n, np.float32),
               radius=np.zeros(n, np.float32), rect=np.zeros((n, 4), np.int32),
               tiles=np.zeros(n, np.int32), canon_abc=np.zeros((n, 3), np.float32),
               canon_mu=np.zeros((n, 2), np.float32), mu2=np.zeros((n, 2)),
               conic=np.zeros((n, 3)), wp=np.zeros((n, 2)), rgb=np.zeros((n, 3)),
               var_terms=np.zeros((n, 2)), comp=np.ones(n))
    fp, dp, ip = c_float, c_double, c_int
    lib().or_project(n, _p(s["means"], dp), _p(s["scales"], dp), _p(s["quats"], dp),
                     _p(s["normals"], dp), _p(s["sh"], dp), _p(s["opac1"], dp), _p(s["opac2"], dp),
                     ctypes.byref(c), ctypes.byref(o), _p(out["mode"], ip), _p(out["depth"], fp), _p(out["radius"], fp),
                     _p(out["rect"], ip), _p(out["tiles"], ip), _p(out["canon_abc"], fp),
                     _p(out["canon_mu"], fp), _p(out["mu2"], dp), _p(out["conic"], dp),
                     _p(out["wp"], dp), _p(out["rgb"], dp), _p(out["var_terms"], dp), _p(out["comp"], dp))
    out["opac1"], out["opac2"] = s["opac1"] * out["comp"], s["opac2"] * out["comp"]
    if errmat:
        out["errmat"] = error_basis(sc, cam, out["mode"], lowpass=lowpass, fov_clamp=fov_clamp, sel=err_sel,
                                    scene64=s)
    return out


def error_basis(sc, cam, mode, lowpass=0.3, fov_clamp=True, sel=None, scene64=None, vectors=False):
    """FP32 error model, shape part: per splat, E = sum_k v_k v_k^T over the 22 inputs of
    the shape terms y = (conic A, B, C, w'x, w'y) (camera-space mean, camera rotation,
    scales, raw quaternion, raw normal), v_k = |x_k| dy/dx_k by central differences in
    FP64: the change of y per unit relative perturbation of x_k.  Returns E [N,15]
    (upper triangle row by row), and with vectors=True also V [N,22,5]."""
    s = scene64 if scene64 is not None else _scene64(sc)
    n = s["means"].shape[0]
    o = make_opts((16, 16), sc.sh_degree, lowpass, False, fov_clamp)
    c = make_camera(cam)
    E = np.zeros((n, 15))
    V = np.zeros((n, 22, 5)) if vectors else None
    mode = np.ascontiguousarray(mode, np.int32)
    selp = None
    if sel is not None:
        sel = np.ascontiguousarray(np.asarray(sel).astype(np.uint8).reshape(n))
        selp = _p(sel, c_ubyte)
    lib().or_error_basis(n, _p(s["means"], c_double), _p(s["scales"], c_double), _p(s["quats"], c_double),
                         _p(s["normals"], c_double), ctypes.byref(c), ctypes.byref(o), _p(mode, c_int), selp,
                         _p(E, c_double), _p(V, c_double) if vectors else None)
    return (E, V) if vectors else E


def pair_bands(proj, ids, px, py, plain=False, mip=False):
    """The FP32 error model's band (a bound on |ln a32 - ln a|, reading B15) and the FP64
    pair weight before the 0.99 clamp, for splats `ids` at pixel centres (px, py);
    band -1 where the exponent is positive."""
    ids = np.ascontiguousarray(ids, np.int32)
    px, py = _d(px).reshape(-1), _d(py).reshape(-1)
    band, a = np.zeros(ids.size), np.zeros(ids.size)
    em = proj.get("errmat")
    em = np.ascontiguousarray(em, np.float64) if em is not None else None
    dp = c_double
    lib().or_pair_bands(int(proj["mode"].shape[0]), _p(np.ascontiguousarray(proj["mode"], np.int32), c_int),
                        _p(_d(proj["mu2"]), dp), _p(_d(proj["conic"]), dp), _p(_d(proj["wp"]), dp),
                        _p(_d(proj["opac1"]), dp), _p(_d(proj["opac2"]), dp), _p(em, dp) if em is not None else None,
                        int(plain), int(mip), ids.size, _p(ids, c_int), _p(px, dp), _p(py, dp), _p(band, dp), _p(a, dp))
    return band, a


def bin_pairs(proj, cam, tile=(16, 16), tile_mask=None):
    """(tile | depth-bits) keys sorted lexicographically with the splat id as tie-break;
    per-tile [start, end) ranges.  Brute force (qsort), not a radix sort."""
    tx, ty = grid(cam, tile)
    n_tiles = tx * ty
    n = proj["tiles"].shape[0]
    mask_p = None
    if tile_mask is not None:
        tile_mask = np.ascontiguousarray(tile_mask, dtype=np.uint8).reshape(n_tiles)
        mask_p = _p(tile_mask, c_ubyte)
    emitted = c_long(0)
    ranges = np.zeros((n_tiles, 2), np.uint32)
    dummy64 = np.zeros(1, np.uint64)
    dummy32 = np.zeros(1, np.uint32)
    total = lib().or_bin(n, _p(proj["tiles"], c_int), _p(proj["rect"], c_int),
                         _p(proj["depth"], c_float), tx, n_tiles, mask_p, 0,
                         _p(dummy64, c_uint64), _p(dummy32, c_uint32), _p(ranges, c_uint32),
                         ctypes.byref(emitted))
    m = int(emitted.value)
    keys = np.zeros(max(m, 1), np.uint64)
    ids = np.zeros(max(m, 1), np.uint32)
    lib().or_bin(n, _p(proj["tiles"], c_int), _p(proj["rect"], c_int),
                 _p(proj["depth"], c_float), tx, n_tiles, mask_p, m,
                 _p(keys, c_uint64), _p(ids, c_uint32), _p(ranges, c_uint32),
                 ctypes.byref(emitted))
    return dict(keys=keys[:m], ids=ids[:m], ranges=ranges, n_pairs=int(total), n_emitted=m)


def render(sc, cam, tile=(16, 16), lowpass=0.3, plain=False, fov_clamp=True, tile_mask=None,
           proj=None, bins=None, rect_mode=0, mip=False, margins=True, composited=False):
    """Forward image: front-to-back compositing of the Eq. 10 pair weights over each
    tile's depth-sorted list (3-sigma tile culling, 1/255 floor, 0.99 clamp, 1e-4 stop).

    Returns image [3,H,W], T [H,W], n_contrib [H,W], margin [H,W] (the smallest relative
    distance of a decision to its threshold), n_comp (composited splats), the
    intermediates proj/bins, and the FP32 error model's verdicts (reading B15):
    margin_a (1/255 floor and step sign), margin_T (1e-4 stop), margin_c (0.99 clamp),
    each the distance to the threshold over the error a binary32 evaluation can carry
    there (<= 1: FP32 cannot be expected to decide it as FP64 does); flip_img, flip_T:
    how far those decisions can move the pixel; touched [N]: splats with such a
    decision in some pixel.  margins=False skips the error model (its outputs are then
    absent): the render alone, as the CPU baseline times it.  composited=True adds
    comp [pairs, tile_h, tile_w] (bool): entry j of the sorted pair list is composited
    at that pixel of its tile (Sec. 3.3 blending: before the stop, at or above the
    1/255 floor)."""
    if proj is None:
        proj = project(sc, cam, tile, lowpass, fov_clamp, rect_mode, mip, errmat=margins)
    if bins is None:
        bins = bin_pairs(proj, cam, tile, tile_mask)
    W, H = int(cam.width), int(cam.height)
    o = make_opts(tile, sc.sh_degree, lowpass, plain, fov_clamp, mip=mip)
    c = make_camera(cam)
    image = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    mg = np.full((H, W), np.inf)
    mga = np.full((H, W), np.inf)
    mgT = np.full((H, W), np.inf)
    ncomp = np.zeros((H, W), np.int32)
    mgc = np.full((H, W), np.inf)
    flip_img = np.zeros((H, W))
    flip_T = np.zeros((H, W))
    n = proj["mode"].shape[0]
    touched = np.zeros(n, np.uint8)
    em = proj.get("errmat")
    if em is not None:
        em = np.ascontiguousarray(em, np.float64)      # kept alive across the call
    em_p = _p(em, c_double) if em is not None else None
    mask_p = None
    if tile_mask is not None:
        tile_mask = np.ascontiguousarray(tile_mask, dtype=np.uint8)
        mask_p = _p(tile_mask, c_ubyte)
    ids = np.ascontiguousarray(bins["ids"], np.uint32)
    if ids.size == 0:
        ids = np.zeros(1, np.uint32)
    dp = c_double
    comp = np.zeros((max(int(bins["ids"].size), 1), tile[1], tile[0]), np.uint8) if composited else None
    lib().or_render_fwd(proj["mode"].shape[0], _p(proj["mode"], c_int), _p(proj["mu2"], dp),
                        _p(proj["conic"], dp), _p(proj["wp"], dp), _p(proj["rgb"], dp),
                        _p(proj["opac1"], dp), _p(proj["opac2"], dp), _p(ids, c_uint32),
                        _p(bins["ranges"], c_uint32), ctypes.byref(c), ctypes.byref(o), mask_p,
                        _p(image, dp), _p(T, dp), _p(nc, c_int), _p(mg, dp),
                        _p(mga, dp) if margins else None, _p(mgT, dp) if margins else None,
                        _p(ncomp, c_int), em_p, *((_p(mgc, dp), _p(flip_img, dp), _p(flip_T, dp), _p(touched, c_ubyte))
                                                  if margins else (None, None, None, None)),
                        _p(comp, c_ubyte) if composited else None)
    extra = dict(comp=comp[:int(bins["ids"].size)].astype(bool)) if composited else {}
    if not margins:
        return dict(image=image, T=T, n_contrib=nc, n_comp=ncomp, proj=proj, bins=bins, **extra)
    return dict(image=image, T=T, n_contrib=nc, margin=mg, margin_a=mga, margin_T=mgT, margin_c=mgc,
                n_comp=ncomp, flip_img=flip_img, flip_T=flip_T, touched=touched.astype(bool),
                proj=proj, bins=bins, **extra)


def rasterize_bwd(sc, cam, dL_dimage, tile=(16, 16), lowpass=0.3, plain=False, fov_clamp=True,
                  tile_mask=None, proj=None, bins=None, mip=False, with_err=False):
    """FP64 adjoint of the compositing alone (Eq. 10 blending, back to front) for the
    loss L = sum(dL_dimage * image): the per-splat screen-space gradients grad2d
    [N,12] (fields G2D_FIELDS; alpha1/alpha2 are the opacities the compositing used).
    with_err: also the FP32 error model's first-order bound on each entry [N,12],
    returned as (grad2d, grad2d_err)."""
    if proj is None:
        proj = project(sc, cam, tile, lowpass, fov_clamp, mip=mip)
    if bins is None:
        bins = bin_pairs(proj, cam, tile, tile_mask)
    n = int(np.asarray(proj["mode"]).shape[0])
    o = make_opts(tile, sc.sh_degree, lowpass, plain, fov_clamp, mip=mip)
    c = make_camera(cam)
    g2 = np.zeros((n, 12))
    g2e = np.zeros((n, 12)) if with_err else None
    em = proj.get("errmat")
    if em is not None:
        em = np.ascontiguousarray(em, np.float64)
    mask_p = None
    if tile_mask is not None:
        tile_mask = np.ascontiguousarray(tile_mask, dtype=np.uint8)
        mask_p = _p(tile_mask, c_ubyte)
    ids = np.ascontiguousarray(bins["ids"], np.uint32)
    if ids.size == 0:
        ids = np.zeros(1, np.uint32)
    dLd = _d(dL_dimage)
    dp = c_double
    lib().or_render_bwd(n, _p(proj["mode"], c_int), _p(proj["mu2"], dp), _p(proj["conic"], dp),
                        _p(proj["wp"], dp), _p(proj["rgb"], dp), _p(proj["opac1"], dp),
                        _p(proj["opac2"], dp), _p(ids, c_uint32), _p(bins["ranges"], c_uint32),
                        ctypes.byref(c), ctypes.byref(o), mask_p, _p(dLd, dp), _p(g2, dp),
                        _p(em, dp) if em is not None else None, _p(g2e, dp) if with_err else None)
    return (g2, g2e) if with_err else g2


def render_bwd(sc, cam, dL_dimage, tile=(16, 16), lowpass=0.3, plain=False, fov_clamp=True,
               tile_mask=None, proj=None, bins=None, mip=False, rect_mode=0):
    """FP64 adjoint of `render` for the loss L = sum(dL_dimage * image).

    Returns the parameter gradients and the per-splat screen-space gradients
    grad2d [N,12] (fields G2D_FIELDS)."""
    if proj is None:
        proj = project(sc, cam, tile, lowpass, fov_clamp, rect_mode, mip)
    if bins is None:
        bins = bin_pairs(proj, cam, tile, tile_mask)
    g2, g2e = rasterize_bwd(sc, cam, dL_dimage, tile, lowpass, plain, fov_clamp, tile_mask, proj, bins, mip,
                            with_err=True)
    grads = project_bwd(sc, cam, proj["mode"], g2, tile, lowpass, fov_clamp, mip)
    grads["grad2d"] = g2
    grads["grad2d_err"] = g2e
    live = np.abs(g2).max(1) > 0
    for k, v in param_error_bound(sc, cam, proj["mode"], g2, g2e, live, tile, lowpass, fov_clamp, mip).items():
        grads["err_" + k] = v
    return grads


# Relative rounding of a binary32 evaluation of the projection adjoint, per input: the
# longest chain of rounded operations from one screen-space gradient entry to a
# parameter gradient is about 32 operations deep.
ADJ_EVAL_ULPS = 32.0
U32 = 2.0 ** -24


def param_error_bound(sc, cam, mode, grad2d, grad2d_err, live=None, tile=(16, 16), lowpass=0.3, fov_clamp=True,
                      mip=False):
    """First-order bound on the error of a binary32 evaluation of the parameter
    gradients: |J|^T (grad2d_err + ADJ_EVAL_ULPS u |grad2d|) per splat, J the Jacobian
    of the projection (parameters -> the 12 screen-space quantities), formed one
    screen-space field at a time with this oracle's FP64 adjoint.  `live` (bool [N])
    restricts the work to splats with a nonzero screen-space gradient."""
    n = int(np.asarray(mode).shape[0])
    m = np.asarray(mode, np.int32).copy()
    if live is not None:
        m[~np.asarray(live, bool)] = CULLED
    x = np.abs(np.asarray(grad2d_err, np.float64)) + ADJ_EVAL_ULPS * U32 * np.abs(np.asarray(grad2d, np.float64))
    out = None
    for f in range(12):
        e = np.zeros((n, 12))
        e[:, f] = x[:, f]
        g = project_bwd(sc, cam, m, e, tile, lowpass, fov_clamp, mip)
        if out is None:
            out = {k: np.abs(v) for k, v in g.items()}
        else:
            for k in out:
                out[k] += np.abs(g[k])
    return out


def project_bwd(sc, cam, mode, grad2d, tile=(16, 16), lowpass=0.3, fov_clamp=True, mip=False):
    """FP64 adjoint of the projection (Eq. 2-5, 7-8, SH colour; with mip, the opacity
    compensation) for given screen-space gradients grad2d [N,12]."""
    s = _scene64(sc)
    n = s["means"].shape[0]
    o = make_opts(tile, sc.sh_degree, lowpass, False, fov_clamp, mip=mip)
    c = make_camera(cam)
    g = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
             normals=np.zeros((n, 3)), opac1=np.zeros(n), opac2=np.zeros(n),
             sh=np.zeros_like(s["sh"]))
    g2 = _d(grad2d)
    mode = np.ascontiguousarray(mode, np.int32)
    dp = c_double
    lib().or_project_bwd(n, _p(s["means"], dp), _p(s["scales"], dp), _p(s["quats"], dp),
                         _p(s["normals"], dp), _p(s["sh"], dp), _p(s["opac1"], dp),
                         _p(s["opac2"], dp), ctypes.byref(c), ctypes.byref(o),
                         _p(mode, c_int), _p(g2, dp), _p(g["means"], dp), _p(g["scales"], dp),
                         _p(g["quats"], dp), _p(g["normals"], dp), _p(g["opac1"], dp),
                         _p(g["opac2"], dp), _p(g["sh"], dp))
    return g


def eval_splat(mean, scale, quat, normal, cam, px, py, lowpass=0.3, fov_clamp=True):
    """hat G and P (= I/2 of Eq. 8) of one splat at pixel positions (px, py)."""
    o = make_opts((16, 16), 0, lowpass, False, fov_clamp)
    c = make_camera(cam)
    px, py = _d(px).reshape(-1), _d(py).reshape(-1)
    G = np.zeros(px.size)
    P = np.zeros(px.size)
    dp = c_double
    mode = lib().or_eval_splat(_p(_d(mean), dp), _p(_d(scale), dp), _p(_d(quat), dp),
                               _p(_d(normal), dp), ctypes.byref(c), ctypes.byref(o), px.size,
                               _p(px, dp), _p(py, dp), _p(G, dp), _p(P, dp))
    return G, P, int(mode)


def sh_eval(deg, dirs):
    """Real SH basis values [n,16] at unit directions [n,3]."""
    dirs = _d(dirs).reshape(-1, 3)
    Y = np.zeros((dirs.shape[0], 16))
    lib().or_sh_eval(int(deg), dirs.shape[0], _p(dirs, c_double), _p(Y, c_double))
    return Y


def render_views(sc, cams, **kw):
    return [render(sc, c, **kw) for c in cams]


def loss_and_grads(sc, cam, dL_dimage, **kw):
    out = render(sc, cam, **kw)
    loss = float(np.sum(out["image"] * _d(dL_dimage)))
    g = render_bwd(sc, cam, dL_dimage, proj=out["proj"], bins=out["bins"],
                   **{k: v for k, v in kw.items() if k != "tile_mask"},
                   tile_mask=kw.get("tile_mask"))
    return loss, g, out


def so_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "liborhgs.so")


def alg1_flat_cov(Sigma, n):
    """Algorithm 1 (Suppl. B.1) in FP64: the covariance of the flattened ellipsoid that
    holds the cut of the Gaussian of covariance Sigma (3x3) by the plane through its
    mean with normal n (3,)."""
    S = _d(Sigma).reshape(9)
    nv = _d(n).reshape(3)
    out = np.zeros(9, np.float64)
    lib().or_alg1_flat_cov(_p(S, c_double), _p(nv, c_double), _p(out, c_double))
    return out.reshape(3, 3)
