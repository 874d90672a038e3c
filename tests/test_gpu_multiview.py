"""Batched multi-view step (one persistent launch sequence over all (view, tile)
items) against one launch sequence per view with gradients accumulated over
views: the images are bitwise identical (each tile's list is the same), the
summed gradients agree to FP32 rounding, and both match the oracle."""
import numpy as np
import pytest

import oracle
from hgs_testutil import check_grads, compare_image, exempt
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def _setup():
    rng = np.random.default_rng(52)
    sc = scenes.scene_uniform(rng, 2500, [-2, -2, -2], [2, 2, 2], -3.4, 0.6, 1.5, 3)
    cams = scenes.fibonacci_cameras(4, radius=6.0, resolutions=[(96, 64), (160, 90), (64, 64), (200, 120)])
    return sc, cams


@pytest.mark.parametrize("tile,batch", [((16, 16), 0), ((8, 8), 64), ((32, 8), 128)])
def test_batched_equals_per_view(cuda_ok, tile, batch):
    import torch
    from paper_2406_02720_b300.multiview import BatchedStep, PerViewStep, packed_upstream
    from paper_2406_02720_b300.rasterizer import Gaussians
    sc, cams = _setup()
    refs = [oracle.render(sc, c, tile=tile) for c in cams]
    from hgs_testutil import masked_upstream
    dL = masked_upstream(scenes.upstream_grad(9, cams), refs)
    g = Gaussians.from_scene(sc)
    b = BatchedStep(cams, g, packed_upstream(dL, "cuda"), tile=tile, batch=batch)
    p = PerViewStep(cams, g, dL, tile=tile, batch=batch)
    for _ in range(2):                       # replay twice: accumulation restarts each step
        b.replay()
        p.replay()
    torch.cuda.synchronize()
    assert b.status() == 0 and p.status() == 0
    for v in range(len(cams)):
        bi = b.images()[v].cpu().numpy()
        pi = p.images()[v].cpu().numpy()
        assert np.array_equal(bi, pi)
        r = b.rast
        compare_image(bi, r.per_pixel(r.final_T)[v].cpu().numpy(), r.per_pixel(r.n_contrib)[v].cpu().numpy(),
                      refs[v], label=f"batched {tile} view {v}")
    tot = None
    for c, d, ref in zip(cams, dL, refs):
        gr = oracle.render_bwd(sc, c, d, tile=tile, proj=ref["proj"], bins=ref["bins"])
        tot = gr if tot is None else {k: tot[k] + gr[k] for k in tot}
    touched = np.logical_or.reduce([r["touched"] for r in refs])
    for k in ("means", "scales", "quats", "normals", "opac1", "opac2", "sh"):
        gb = getattr(b.grads, k).cpu().numpy().astype(np.float64)
        gp = getattr(p.grads, k).cpu().numpy().astype(np.float64)
        # float atomics sum in a different order in the two paths
        np.testing.assert_allclose(gb, gp, rtol=1e-3, atol=1e-5 * np.abs(gp).max())
        check_grads(gb, tot[k], touched, label=f"batched {tile} {k}", err=tot["err_" + k])


def test_many_views_pairs_equal_per_view_launches(cuda_ok):
    """4.5M (view, splat) entries in one launch sequence (the pair-offset scan then runs
    over more than 2048 groups of 8 chunks: the 16-row scan) give exactly the
    sorted pairs of five single-view launches (each pinned against the oracle's sort
    elsewhere), with tile ids offset by view and splat ids by n * view."""
    from paper_2406_02720_b300 import hgs as H
    from paper_2406_02720_b300.rasterizer import Gaussians, Rasterizer
    rng = np.random.default_rng(61)
    n = 900_000
    sc = scenes.scene_uniform(rng, n, [-2, -2, -2], [2, 2, 2], -4.6, 0.5, 1.5, 0)
    cams = scenes.fibonacci_cameras(5, radius=6.0, resolutions=[(320, 240), (256, 192), (320, 180), (200, 200),
                                                               (288, 216)])
    g = Gaussians.from_scene(sc)
    cfg = H.make_config()
    batched = Rasterizer(cams, n, cfg, keep_keys=True)
    batched.forward(g)
    bk, bi = (x.cpu().numpy() for x in batched.sorted_pairs())
    bk, bi = bk.view(np.uint64), bi.view(np.uint32)
    assert batched.read_status() == 0
    assert -(-len(cams) * n // 2048) > 2048             # more scan groups than the 2-row scan holds
    off = 0
    parts_k, parts_i = [], []
    for v, cam in enumerate(cams):
        r = Rasterizer([cam], n, cfg, keep_keys=True)
        r.forward(g)
        k, i = (x.cpu().numpy() for x in r.sorted_pairs())
        k, i = k.view(np.uint64), i.view(np.uint32)
        parts_k.append(k + (np.uint64(off) << np.uint64(32)))
        parts_i.append(i + np.uint32(v * n))
        tx, ty = oracle.grid(cam, (16, 16))
        off += tx * ty
    assert np.array_equal(bk, np.concatenate(parts_k))
    assert np.array_equal(bi, np.concatenate(parts_i))


def test_maximum_view_count(cuda_ok):
    """HGS_MAX_VIEWS (256) cameras of uneven small sizes in one launch sequence: every
    view's image matches the oracle's render of that view alone."""
    from paper_2406_02720_b300 import hgs as H
    from paper_2406_02720_b300.rasterizer import Gaussians, Rasterizer
    rng = np.random.default_rng(63)
    sc = scenes.scene_uniform(rng, 400, [-2, -2, -2], [2, 2, 2], -3.0, 0.5, 1.5, 1)
    sizes = [(16, 16), (24, 16), (40, 24), (17, 33)]
    cams = scenes.fibonacci_cameras(H.HGS_MAX_VIEWS, radius=6.0, resolutions=sizes)
    g = Gaussians.from_scene(sc)
    r = Rasterizer(cams, sc.n, H.make_config())
    r.forward(g)
    assert r.read_status() == 0
    imgs = [x.cpu().numpy() for x in r.images()]
    for v in list(range(0, H.HGS_MAX_VIEWS, 17)) + [H.HGS_MAX_VIEWS - 1]:
        ref = oracle.render(sc, cams[v])
        ok = ~exempt(ref)
        assert np.abs(imgs[v] - ref["image"])[:, ok].max() <= 1e-4, v
