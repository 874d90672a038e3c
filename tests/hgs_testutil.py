"""Shared helpers for the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

import oracle

# A pixel whose oracle decisions (1/255 floor, step-mode sign) sit within this
# relative distance of their threshold can flip between FP32 and FP64.  The
# oracle's margin_a / margin_T are this distance divided by the error a binary32
# evaluation can carry (which includes the binary32 position of the splat and,
# for the 1e-4 stop, the errors of every composited splat); <= 1 means exempt.
EXEMPT_MARGIN = 1e-4


def exempt(ref):
    """Pixels whose threshold decisions FP32 cannot be expected to reproduce."""
    if "margin_a" not in ref:
        return ref["margin"] <= EXEMPT_MARGIN
    return (ref["margin_a"] <= 1.0) | (ref["margin_T"] <= 1.0)


IMAGE_ATOL = 1e-4
# One threshold flip changes a pixel by at most about a/255-scale amounts; exempt
# pixels must still agree to this bound.
EXEMPT_ATOL = 2e-2


def gpu_render(sc, cams, tile=(16, 16), batch=0, lowpass=0.3, plain=False, persistent=True,
               pair_capacity=None, dL=None, rect_mode=0, mip=False):
    import torch
    from paper_2406_02720_b300 import hgs as H
    from paper_2406_02720_b300.rasterizer import Gaussians, Rasterizer
    cfg = H.make_config(tile=tile, batch=batch, lowpass=lowpass, plain=plain, persistent=persistent,
                        rect_mode=rect_mode, mip=mip)
    g = Gaussians.from_scene(sc)
    r = Rasterizer(cams, sc.n, cfg, pair_capacity=pair_capacity, keep_keys=True)
    r.forward(g)
    out = dict(rast=r, g=g)
    out["images"] = [x.cpu().numpy() for x in r.images()]
    out["T"] = [x.cpu().numpy() for x in r.per_pixel(r.final_T)]
    out["n_contrib"] = [x.cpu().numpy() for x in r.per_pixel(r.n_contrib)]
    k, i = r.sorted_pairs()
    out["keys"] = k.cpu().numpy().view(np.uint64)
    out["ids"] = i.cpu().numpy().view(np.uint32)
    out["ranges"] = r.ranges.cpu().numpy().view(np.uint32)
    out["rec"] = r.rec.cpu().numpy().reshape(len(cams), sc.n, 16)
    out["depth"] = r.depth.cpu().numpy().reshape(len(cams), sc.n)
    out["rect"] = r.rect.cpu().numpy().reshape(len(cams), sc.n, 4)
    out["tiles"] = r.tiles.cpu().numpy().reshape(len(cams), sc.n)
    fl = r.fp64_list.cpu().numpy().view(np.uint32)
    out["fp64_fwd"] = np.sort(fl[1:1 + fl[0]])       # (view, splat) records given the FP64 half-plane path
    if dL is not None:
        flat = np.concatenate([np.asarray(d, np.float32).reshape(-1) for d in dL])
        dl = torch.from_numpy(flat).cuda()
        gr = r.backward(g, dl)
        out["grads"] = {k2: getattr(gr, k2).cpu().numpy().astype(np.float64) for k2 in
                        ("means", "scales", "quats", "normals", "opac1", "opac2", "sh")}
        out["grad2d"] = r.grad2d.cpu().numpy().reshape(len(cams), sc.n, 12)
    torch.cuda.synchronize()
    return out


def compare_image(gpu_img, gpu_T, gpu_nc, ref, atol=IMAGE_ATOL, max_exempt_frac=5e-2):
    """Max-abs image/T error on pixels away from threshold decisions; n_contrib equal there.
    Pixels with a decision within EXEMPT_MARGIN of its threshold (long lists make
    hundreds of decisions per pixel) are held to EXEMPT_ATOL only."""
    ok = ~exempt(ref)
    n_ex = int((~ok).sum())
    assert n_ex <= max(4, max_exempt_frac * ok.size), f"{n_ex} exempt pixels of {ok.size}"
    if n_ex:
        ex_err = np.abs(gpu_img.astype(np.float64) - ref["image"])[:, ~ok]
        assert ex_err.max() <= EXEMPT_ATOL, f"exempt pixel error {ex_err.max():.3g}"
    err = np.abs(gpu_img.astype(np.float64) - ref["image"])[:, ok]
    terr = np.abs(gpu_T.astype(np.float64) - ref["T"])[ok]
    assert err.size == 0 or err.max() <= atol, f"image max abs err {err.max():.3g}"
    assert terr.size == 0 or terr.max() <= atol, f"T max abs err {terr.max():.3g}"
    assert np.array_equal(gpu_nc[ok], ref["n_contrib"][ok])
    return dict(max_err=float(err.max()) if err.size else 0.0, exempt=n_ex)


def grad_close(g, ref, rel=1e-3, floor_frac=1e-3):
    """|g - ref| <= rel * max(|ref|, floor_frac * max|ref|) elementwise."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), floor_frac * max(np.abs(ref).max(), 1e-30))
    bad = np.abs(g - ref) > rel * scale
    return bad, scale


def masked_upstream(dL_list, refs):
    """dL/dimage with exempt pixels zeroed (both sides get the same array)."""
    out = []
    for d, r in zip(dL_list, refs):
        d = np.array(d, np.float32, copy=True)
        d[:, exempt(r)] = 0.0
        out.append(d)
    return out
