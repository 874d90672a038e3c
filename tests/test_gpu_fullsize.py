"""Parity at the full benchmark size (3M half-Gaussians, 1920x1080, 16x16 tiles,
256-splat batches: the launch configuration bench.py times), on outputs the
FP64 oracle can compute piecewise: the total pair count, the sorted pairs and
ranges of sampled tiles, the image of sampled tile blocks, and the gradients of
splats that lie entirely inside those blocks."""
import numpy as np
import pytest

import oracle
from hgs_testutil import compare_image, exempt, grad_close
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def _blocks(tx, ty, ranges, rng, n_random=8, n_dense=4, size=3):
    lens = (ranges[:, 1].astype(np.int64) - ranges[:, 0]).reshape(ty, tx)
    centres = [(int(rng.integers(1, ty - 1)), int(rng.integers(1, tx - 1))) for _ in range(n_random)]
    for flat in np.argsort(lens.ravel())[::-1][:n_dense]:
        centres.append((int(flat // tx), int(flat % tx)))
    mask = np.zeros((ty, tx), np.uint8)
    for cy, cx in centres:
        mask[max(cy - 1, 0):cy - 1 + size, max(cx - 1, 0):cx - 1 + size] = 1
    return mask.ravel()


def test_config3_sampled_parity(cuda_ok):
    import torch
    from paper_2406_02720_b300 import hgs as H
    from paper_2406_02720_b300.rasterizer import Gaussians, Rasterizer
    sc, cams = scenes.config3()
    cam = cams[0]
    W, Hh = cam.width, cam.height
    cfg = H.make_config(tile=(16, 16), batch=0)
    g = Gaussians.from_scene(sc)
    r = Rasterizer(cams, sc.n, cfg, keep_keys=True)
    r.forward(g)
    ranges = r.ranges.cpu().numpy().view(np.uint32)
    keys = r.keys[:int(r.num_pairs.item())].cpu().numpy().view(np.uint64)
    ids = r.ids[:int(r.num_pairs.item())].cpu().numpy().view(np.uint32)
    img = r.images()[0].cpu().numpy()
    T = r.per_pixel(r.final_T)[0].cpu().numpy()
    nc = r.per_pixel(r.n_contrib)[0].cpu().numpy()
    tx, ty = oracle.grid(cam, (16, 16))
    mask = _blocks(tx, ty, ranges, np.random.default_rng(17))

    pr = oracle.project(sc, cam)
    bins = oracle.bin_pairs(pr, cam, tile_mask=mask)
    assert bins["n_pairs"] == keys.size              # every pair of the frame, bit-exact count
    for t in np.flatnonzero(mask):
        a, b = ranges[t]
        ra, rb = bins["ranges"][t]
        assert b - a == rb - ra
        assert np.array_equal(keys[a:b], bins["keys"][ra:rb])
        assert np.array_equal(ids[a:b], bins["ids"][ra:rb])
    ref = oracle.render(sc, cam, tile_mask=mask, proj=pr, bins=bins)
    pix = np.kron(mask.reshape(ty, tx), np.ones((16, 16), np.uint8))[:Hh, :W].astype(bool)
    sub = dict(image=ref["image"][:, pix][:, None, :], T=ref["T"][pix][None], n_contrib=ref["n_contrib"][pix][None],
               margin=ref["margin"][pix][None], margin_a=ref["margin_a"][pix][None],
               margin_T=ref["margin_T"][pix][None], n_comp=ref["n_comp"][pix][None])
    compare_image(img[:, pix][:, None, :], T[pix][None], nc[pix][None], sub)
    assert ref["n_contrib"][pix].max() > 50        # dense lists are part of the sample

    # gradients of the splats whose rect lies inside the sampled blocks
    dL = scenes.upstream_grad(103, cams)[0].copy()
    dL[:, pix & exempt(ref)] = 0.0
    grads = r.backward(g, torch.from_numpy(dL.reshape(-1)).cuda())
    gref = oracle.render_bwd(sc, cam, dL, tile_mask=mask, proj=pr, bins=bins)
    m2 = mask.reshape(ty, tx)
    inside = []
    for i in np.flatnonzero(pr["tiles"] > 0):
        x0, y0, x1, y1 = pr["rect"][i]
        if m2[y0:y1, x0:x1].all():
            inside.append(i)
    inside = np.array(inside)
    assert inside.size > 200
    g2 = r.grad2d.cpu().numpy()[inside]
    bad, _ = grad_close(g2, gref["grad2d"][inside])
    assert bad.mean() < 2e-3, bad.sum()
    for k in ("means", "scales", "quats", "normals", "opac1", "opac2", "sh"):
        got = getattr(grads, k).cpu().numpy().astype(np.float64)[inside]
        bad, _ = grad_close(got, gref[k][inside])
        assert bad.mean() < 2e-3, (k, int(bad.sum()), bad.size)
