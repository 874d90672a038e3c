"""Parity at workload scale, on outputs the FP64 oracle can compute piecewise.

Config 3 (3M half-Gaussians, 1920x1080: the launch configuration bench.py times),
four cameras of config 4 (1M splats, 640x360 to 1920x1080) through the batched
multi-view step, and config 5 at its largest point (6M splats with grazing 100:1
disks).  Per view a set of 3x3-tile blocks is sampled (random ones and the
densest ones, chosen from the oracle's own per-tile pair counts).  Checked: the
total pair count; the sorted pairs and range lengths of every sampled tile
(bit-exact); the image, final T and n_contrib of every sampled pixel (the bars of
hgs_testutil.compare_image); and the gradients of every splat and every (view,
splat) record, with the upstream gradient zero outside the sampled blocks, so that
both sides sum the same pixels."""
import numpy as np
import pytest

import oracle
from hgs_testutil import MAX_EXEMPT_FRAC_DENSE, check_grads, compare_image, grad_exempt
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu

TILE = 16
FIELDS = ("means", "scales", "quats", "normals", "opac1", "opac2", "sh")


def tile_counts(pr, cam):
    """Pairs per tile from the oracle's tile rects (a 2-D difference array)."""
    tx, ty = oracle.grid(cam, (TILE, TILE))
    diff = np.zeros((ty + 1, tx + 1), np.int64)
    live = pr["tiles"] > 0
    x0, y0, x1, y1 = (pr["rect"][live, k] for k in range(4))
    np.add.at(diff, (y0, x0), 1)
    np.add.at(diff, (y0, x1), -1)
    np.add.at(diff, (y1, x0), -1)
    np.add.at(diff, (y1, x1), 1)
    return diff.cumsum(0).cumsum(1)[:ty, :tx]


def sample_blocks(counts, rng, n_random=8, n_dense=4):
    ty, tx = counts.shape
    centres = [(int(rng.integers(1, ty - 1)), int(rng.integers(1, tx - 1))) for _ in range(n_random)]
    for flat in np.argsort(counts.ravel(), kind="stable")[::-1][:n_dense]:
        centres.append((int(flat // tx), int(flat % tx)))
    mask = np.zeros((ty, tx), np.uint8)
    for cy, cx in centres:
        mask[max(cy - 1, 0):cy + 2, max(cx - 1, 0):cx + 2] = 1
    return mask.ravel()


def oracle_views(sc, cams, seed):
    """Per view: projection, sampled tile mask, binning and render of the sampled tiles,
    and dL/dimage ~ N(0,1) zeroed outside them and on gradient-exempt pixels."""
    rng = np.random.default_rng(seed)
    dLs = scenes.upstream_grad(seed + 100, cams)
    views = []
    for cam, dL in zip(cams, dLs):
        tx, ty = oracle.grid(cam, (TILE, TILE))
        pr = oracle.project(sc, cam, errmat=False)
        mask = sample_blocks(tile_counts(pr, cam), rng)
        bins = oracle.bin_pairs(pr, cam, tile_mask=mask)
        sel = np.zeros(sc.n, bool)
        sel[bins["ids"]] = True
        pr["errmat"] = oracle.error_basis(sc, cam, pr["mode"], sel=sel)
        ref = oracle.render(sc, cam, tile_mask=mask, proj=pr, bins=bins)
        pix = np.kron(mask.reshape(ty, tx), np.ones((TILE, TILE), np.uint8))[:cam.height, :cam.width].astype(bool)
        dL = dL.copy()
        dL[:, ~pix | grad_exempt(ref)] = 0.0
        views.append(dict(cam=cam, pr=pr, mask=mask, bins=bins, ref=ref, pix=pix, dL=dL, tiles=tx * ty))
    return views


def check_sampled(sc, views, ranges, ids, n_pairs, images, Ts, ncs, grads, grad2d, label):
    tile_off = 0
    for v, w in enumerate(views):
        rv = ranges[tile_off:tile_off + w["tiles"]]
        bins = w["bins"]
        assert n_pairs[v] == bins["n_pairs"], f"{label} view {v}: pair count"
        for t in np.flatnonzero(w["mask"]):
            a, b = rv[t]
            ra, rb = bins["ranges"][t]
            assert b - a == rb - ra, f"{label} view {v} tile {t}: list length"
            assert np.array_equal(ids[a:b] - np.uint32(v * sc.n), bins["ids"][ra:rb]), f"{label} view {v} tile {t}"
        pix = w["pix"]
        compare_image(images[v][:, pix], Ts[v][pix], ncs[v][pix], w["ref"], pix=pix,
                      max_exempt_frac=MAX_EXEMPT_FRAC_DENSE, label=f"{label} view {v}")
        assert w["ref"]["n_contrib"][pix].max() > 50            # dense lists are part of the sample
        tile_off += w["tiles"]
    tot, touched = None, np.zeros(sc.n, bool)
    for v, w in enumerate(views):
        g = oracle.render_bwd(sc, w["cam"], w["dL"], tile_mask=w["mask"], proj=w["pr"], bins=w["bins"])
        nm = w["pr"]["mode"] == oracle.NORMAL
        check_grads(grad2d[v][nm], g["grad2d"][nm], w["ref"]["touched"][nm], label=f"{label} view {v} grad2d",
                    err=g["grad2d_err"][nm])
        tot = g if tot is None else {k: tot[k] + g[k] for k in tot}
        touched |= w["ref"]["touched"]
    for k in FIELDS:
        assert np.abs(tot[k]).max() > 0
        check_grads(grads[k], tot[k], touched, label=f"{label} {k}", err=tot["err_" + k])


def run_single_view(sc, cams, seed, label):
    import torch
    from paper_2406_02720_b300 import hgs as H
    from paper_2406_02720_b300.rasterizer import Gaussians, Rasterizer
    views = oracle_views(sc, cams, seed)
    g = Gaussians.from_scene(sc)
    r = Rasterizer(cams, sc.n, H.make_config(tile=(TILE, TILE)))
    r.forward(g)
    gr = r.backward(g, torch.from_numpy(views[0]["dL"].reshape(-1)).cuda())
    torch.cuda.synchronize()
    assert r.read_status() == 0
    n = int(r.num_pairs.item())
    check_sampled(sc, views, r.ranges.cpu().numpy().view(np.uint32), r.ids[:n].cpu().numpy().view(np.uint32), [n],
                  [x.cpu().numpy() for x in r.images()], [x.cpu().numpy() for x in r.per_pixel(r.final_T)],
                  [x.cpu().numpy() for x in r.per_pixel(r.n_contrib)],
                  {k: getattr(gr, k).cpu().numpy().astype(np.float64) for k in FIELDS},
                  [r.grad2d.cpu().numpy().reshape(sc.n, 12)], label)


def test_config3_sampled_parity(cuda_ok):
    sc, cams = scenes.config3()
    run_single_view(sc, cams, 17, "config3")


def test_config5_largest_point_sampled_parity(cuda_ok):
    """6M splats, 30% grazing 100:1 disks (the top of the stress sweep bench.py times)."""
    sc, cams = scenes.config5(n=6_000_000)
    run_single_view(sc, cams, 20, "config5 6M")


def test_config4_four_views_batched_sampled_parity(cuda_ok):
    """Four of config 4's 64 cameras, one of each resolution, rendered in one batched
    step (one launch sequence over the global (view, tile) queue, replayed as a CUDA
    graph), against the oracle's render of each view alone."""
    import torch
    from paper_2406_02720_b300.multiview import BatchedStep, packed_upstream
    from paper_2406_02720_b300.rasterizer import Gaussians
    sc, cams64 = scenes.config4()
    cams = [cams64[i] for i in (1, 2, 5, 8)]
    assert sorted((c.width, c.height) for c in cams) == sorted(scenes.RESOLUTIONS)
    views = oracle_views(sc, cams, 19)
    g = Gaussians.from_scene(sc)
    step = BatchedStep(cams, g, packed_upstream([w["dL"] for w in views], "cuda"))
    step.replay()
    torch.cuda.synchronize()
    assert step.status() == 0
    r = step.rast
    n = int(r.num_pairs.item())
    ranges = r.ranges.cpu().numpy().view(np.uint32)
    ids = r.ids[:n].cpu().numpy().view(np.uint32)
    # pair counts per view from the global ranges (the tiles of view v are contiguous)
    counts, off = [], 0
    for w in views:
        rv = ranges[off:off + w["tiles"]]
        counts.append(int((rv[:, 1].astype(np.int64) - rv[:, 0]).sum()))
        off += w["tiles"]
    assert sum(counts) == n
    g2 = r.grad2d.cpu().numpy().reshape(len(cams), sc.n, 12)
    check_sampled(sc, views, ranges, ids, counts, [x.cpu().numpy() for x in step.images()],
                  [x.cpu().numpy() for x in r.per_pixel(r.final_T)], [x.cpu().numpy() for x in r.per_pixel(r.n_contrib)],
                  {k: getattr(step.grads, k).cpu().numpy().astype(np.float64) for k in FIELDS},
                  [g2[v] for v in range(len(cams))], "config4")
