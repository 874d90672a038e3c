"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars: sort order, tile ranges, depth keys and tile rects bit-exact; images and
final transmittance within 1e-4 max-abs on every pixel none of whose threshold
decisions lies within the oracle's FP32 error band (reading B15), n_contrib
equal there, the others within 1e-4 plus the change their decisions can cause,
and at most 0.1% of pixels exempt; gradients within 1e-3 relative (floor 1e-3
of the tensor's largest entry) of the FP64 adjoint, with the upstream gradient
zeroed on the exempt pixels, except at most 0.1% of entries, each within 1e-2
and on a splat with a marked decision.
"""
import ctypes

import numpy as np
import pytest

import oracle
from hgs_testutil import check_grads, compare_image, exempt, gpu_render, masked_upstream
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def _ragged_scene(seed=21, n=1500):
    rng = np.random.default_rng(seed)
    sc = scenes.scene_uniform(rng, n, [-1.6, -1.2, 2], [1.6, 1.2, 7], -3.0, 0.6, 1.2, 1)
    return sc, [scenes.identity_camera(100, 75, 70.0, 51.0, 36.5, bg=(0.1, 0.2, 0.3))]


@pytest.fixture(scope="module")
def cfg1():
    return scenes.config1()


def test_projection_fields(cuda_ok, cfg1):
    sc, cams = cfg1
    out = gpu_render(sc, cams)
    pr = oracle.project(sc, cams[0])
    assert np.array_equal(out["tiles"][0], pr["tiles"].astype(np.int32))
    vis = pr["tiles"] > 0
    assert np.array_equal(out["depth"][0].view(np.uint32), pr["depth"].view(np.uint32))
    assert np.array_equal(out["rect"][0][vis], pr["rect"][vis])
    rec = out["rec"][0].astype(np.float64)
    # centre = integer anchor + remainder, to ~1e-7 px of the FP64 centre
    assert np.all(rec[vis, 0:2] == np.round(rec[vis, 0:2]))
    mu = rec[vis, 0:2] + rec[vis, 2:4]
    assert np.abs(mu - pr["mu2"][vis]).max() < 2e-7        # the FP32 error model's centre bound
    assert np.abs(mu - pr["canon_mu"][vis]).max() < 1e-3      # and close to the binning centre
    u11, u12, u22 = rec[vis, 4], rec[vis, 5], rec[vis, 6]
    Q = np.stack([u11 * u11, u11 * u12, u12 * u12 + u22 * u22], 1)     # conic = U^T U
    Qr = pr["conic"][vis]
    assert np.all(np.abs(Q - Qr).max(1) <= 2e-6 * np.abs(Qr).max(1))
    normal = pr["mode"][vis] == oracle.NORMAL
    wp = rec[vis, 7:9][normal]
    wr = pr["wp"][vis][normal]
    assert np.all(np.abs(wp - wr).max(1) <= 1e-4 * np.maximum(np.abs(wr).max(1), 1e-3))
    np.testing.assert_allclose(rec[vis, 11:14], pr["rgb"][vis], atol=2e-6)
    np.testing.assert_array_equal(rec[vis, 9], sc.opac1[vis])
    np.testing.assert_array_equal(rec[vis, 10], sc.opac2[vis])


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_binning_bit_exact(cuda_ok, tile):
    sc, cams = _ragged_scene()
    out = gpu_render(sc, cams, tile=tile)
    ref = oracle.bin_pairs(oracle.project(sc, cams[0], tile=tile), cams[0], tile)
    assert out["keys"].size == ref["n_pairs"] > 1000
    assert np.array_equal(out["keys"], ref["keys"])
    assert np.array_equal(out["ids"], ref["ids"])
    assert np.array_equal(out["ranges"], ref["ranges"])


@pytest.mark.parametrize("tile,batch", [((16, 16), 0), ((8, 8), 32), ((32, 8), 128), ((16, 16), 64),
                                        ((16, 16), 512)])
def test_forward_image_ragged(cuda_ok, tile, batch):
    sc, cams = _ragged_scene()
    out = gpu_render(sc, cams, tile=tile, batch=batch)
    ref = oracle.render(sc, cams[0], tile=tile)
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label=f"ragged {tile} b{batch}")
    assert ref["n_contrib"].max() > 5


def test_forward_config1(cuda_ok, cfg1):
    sc, cams = cfg1
    out = gpu_render(sc, cams)
    ref = oracle.render(sc, cams[0])
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="config1")
    assert (ref["T"] < 0.01).mean() > 0.01      # early termination happens in this scene


def test_equal_opacity_is_bitwise_plain_3dgs(cuda_ok):
    sc, cams = _ragged_scene(seed=5)
    sc.opac2[:] = sc.opac1
    a = gpu_render(sc, cams)
    b = gpu_render(sc, cams, plain=True)
    assert np.array_equal(a["images"][0], b["images"][0])
    assert np.array_equal(a["n_contrib"][0], b["n_contrib"][0])
    rng = np.random.default_rng(3)
    dL = [rng.standard_normal((3, 75, 100)).astype(np.float32)]
    ga = gpu_render(sc, cams, dL=dL)["grads"]
    assert np.all(ga["normals"] == 0.0)


def test_plain_mode_against_oracle(cuda_ok):
    """hgs_config.plain = 1 renders plain 3D-GS (alpha = alpha1 G) from the same records:
    image and gradients against the oracle's plain mode, on a scene whose half opacities
    differ (so the flag visibly changes the image)."""
    rng = np.random.default_rng(37)
    sc = scenes.scene_uniform(rng, 800, [-1.3, -0.8, 2.5], [1.3, 0.8, 6], -3.3, 0.5, 1.5, 3)
    cams = [scenes.identity_camera(160, 96, 90.0, 80.0, 48.0, bg=(0.3, 0.2, 0.1))]
    ref = oracle.render(sc, cams[0], plain=True)
    half = oracle.render(sc, cams[0])
    assert np.abs(half["image"] - ref["image"]).max() > 1e-2
    dL = masked_upstream(scenes.upstream_grad(103, cams), [ref])
    out = gpu_render(sc, cams, plain=True, dL=dL)
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="plain mode")
    gref = oracle.render_bwd(sc, cams[0], dL[0], plain=True, proj=ref["proj"], bins=ref["bins"])
    assert np.all(out["grads"]["opac2"] == 0.0) and np.all(out["grads"]["normals"] == 0.0)
    for k in ("means", "scales", "quats", "opac1", "sh"):
        check_grads(out["grads"][k], gref[k], ref["touched"], label=f"plain mode {k}", err=gref["err_" + k])


def test_complement_symmetry(cuda_ok):
    sc, cams = _ragged_scene(seed=6)
    b = scenes.Scene(sc.means, sc.scales, sc.quats, -sc.normals, sc.opac2.copy(), sc.opac1.copy(), sc.sh,
                     sc.sh_degree)
    ra, rb = gpu_render(sc, cams), gpu_render(b, cams)
    ref = oracle.render(sc, cams[0])
    ok = ~exempt(ref)
    assert np.abs(ra["images"][0] - rb["images"][0])[:, ok].max() <= 1e-6


def test_gradients_against_fp64_adjoint(cuda_ok):
    rng = np.random.default_rng(31)
    sc = scenes.scene_uniform(rng, 800, [-1.3, -0.8, 2.5], [1.3, 0.8, 6], -3.3, 0.5, 1.5, 3)
    cams = [scenes.identity_camera(160, 96, 90.0, 80.0, 48.0, bg=(0.3, 0.2, 0.1))]
    ref = oracle.render(sc, cams[0])
    dL = masked_upstream(scenes.upstream_grad(102, cams), [ref])
    out = gpu_render(sc, cams, dL=dL)
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="gradient scene")
    gref = oracle.render_bwd(sc, cams[0], dL[0], proj=ref["proj"], bins=ref["bins"])
    # screen-space gradients first (compositing adjoint), then parameters
    g2 = out["grad2d"][0]
    vis = ref["proj"]["mode"] == oracle.NORMAL
    check_grads(g2[vis], gref["grad2d"][vis], ref["touched"][vis], label="grad2d", err=gref["grad2d_err"][vis])
    for k in ("means", "scales", "quats", "normals", "opac1", "opac2", "sh"):
        check_grads(out["grads"][k], gref[k], ref["touched"], label=k, err=gref["err_" + k])


@pytest.mark.parametrize("tile,batch,persistent", [((8, 8), 32, True), ((32, 8), 128, False),
                                                    ((32, 8), 512, True), ((16, 16), 64, False)])
def test_gradients_other_tiles_and_batches(cuda_ok, tile, batch, persistent):
    """The adjoint in every tile shape the autotuner may pick, with batches that split
    each list into several staged rounds, per-tile and persistent launches."""
    rng = np.random.default_rng(33)
    sc = scenes.scene_uniform(rng, 900, [-1.4, -0.9, 2.5], [1.4, 0.9, 6], -3.3, 0.5, 1.5, 2)
    cams = [scenes.identity_camera(150, 90, 85.0, 75.0, 45.0, bg=(0.2, 0.1, 0.3))]
    ref = oracle.render(sc, cams[0], tile=tile)
    dL = masked_upstream(scenes.upstream_grad(104, cams), [ref])
    out = gpu_render(sc, cams, tile=tile, batch=batch, persistent=persistent, dL=dL)
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label=f"gradients {tile} b{batch}")
    gref = oracle.render_bwd(sc, cams[0], dL[0], tile=tile, proj=ref["proj"], bins=ref["bins"])
    vis = ref["proj"]["mode"] == oracle.NORMAL
    check_grads(out["grad2d"][0][vis], gref["grad2d"][vis], ref["touched"][vis], label=f"grad2d {tile}",
                err=gref["grad2d_err"][vis])
    for k in ("means", "scales", "quats", "normals", "opac1", "opac2", "sh"):
        check_grads(out["grads"][k], gref[k], ref["touched"], label=f"{k} {tile} b{batch}", err=gref["err_" + k])


def test_multiview_persistent_matches_per_tile_launch(cuda_ok):
    rng = np.random.default_rng(41)
    sc = scenes.scene_uniform(rng, 3000, [-2, -2, -2], [2, 2, 2], -3.5, 0.6, 1.5, 2)
    sizes = [(120, 72), (64, 48), (200, 110)]
    cams = []
    for k, (w, h) in enumerate(sizes):
        c = scenes.fibonacci_cameras(3, radius=6.0, resolutions=[(w, h)])[k]
        cams.append(c)
    a = gpu_render(sc, cams, persistent=False)
    b = gpu_render(sc, cams, persistent=True)
    for v in range(3):
        assert np.array_equal(a["images"][v], b["images"][v])
        assert np.array_equal(a["n_contrib"][v], b["n_contrib"][v])
    # each view against its own oracle run
    for v, cam in enumerate(cams):
        ref = oracle.render(sc, cam)
        compare_image(b["images"][v], b["T"][v], b["n_contrib"][v], ref, label=f"multi-view {v}")
    # global sort: the keys of view v are the oracle keys shifted by the view's tile offset
    off = 0
    for v, cam in enumerate(cams):
        tx, ty = oracle.grid(cam, (16, 16))
        ref = oracle.bin_pairs(oracle.project(sc, cam), cam)
        sel = (b["keys"] >> np.uint64(32)) - np.uint64(off)
        m = (b["keys"] >> np.uint64(32) >= off) & (b["keys"] >> np.uint64(32) < off + tx * ty)
        want = ref["keys"] + (np.uint64(off) << np.uint64(32))
        assert np.array_equal(b["keys"][m], want)
        assert np.array_equal(b["ids"][m], ref["ids"] + np.uint32(v * sc.n))
        off += tx * ty


def test_multiview_gradients_sum_over_views(cuda_ok):
    rng = np.random.default_rng(43)
    sc = scenes.scene_uniform(rng, 600, [-1.5, -1.5, -1.5], [1.5, 1.5, 1.5], -3.2, 0.5, 1.5, 1)
    cams = scenes.fibonacci_cameras(2, radius=5.0, resolutions=[(96, 64)])
    refs = [oracle.render(sc, c) for c in cams]
    dL = masked_upstream(scenes.upstream_grad(7, cams), refs)
    out = gpu_render(sc, cams, dL=dL, persistent=True)
    tot = None
    for c, d, r in zip(cams, dL, refs):
        g = oracle.render_bwd(sc, c, d, proj=r["proj"], bins=r["bins"])
        tot = g if tot is None else {k: tot[k] + g[k] for k in tot}
    touched = np.logical_or.reduce([r["touched"] for r in refs])
    for k in ("means", "scales", "quats", "normals", "opac1", "opac2", "sh"):
        check_grads(out["grads"][k], tot[k], touched, label=f"two views {k}", err=tot["err_" + k])


def test_capacity_overflow_sets_status_and_count(cuda_ok):
    import torch
    from paper_2406_02720_b300 import hgs as H
    from paper_2406_02720_b300.rasterizer import Gaussians, Rasterizer
    sc, cams = scenes.config1()
    r = Rasterizer(cams, sc.n, H.make_config(), pair_capacity=100, keep_keys=True)
    g = Gaussians.from_scene(sc)
    r.clear_status()
    r.project(g)
    r.bin()
    st = r.read_status()
    ref = oracle.bin_pairs(oracle.project(sc, cams[0]), cams[0])
    assert st & H.HGS_DEV_CAPACITY
    assert int(r.num_pairs.item()) == ref["n_pairs"]
    # the high-level forward grows the buffer and succeeds
    r.forward(g)
    assert r.capacity >= ref["n_pairs"]
    k, i = r.sorted_pairs()
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ref["keys"])
    torch.cuda.synchronize()


def test_empty_and_all_culled(cuda_ok):
    sc, cams = scenes.config1()
    behind = sc.subset(np.arange(50))
    behind.means[:, 2] = -3.0                      # behind the camera: all culled
    out = gpu_render(behind, cams)
    assert out["keys"].size == 0
    assert np.all(out["images"][0] == 0.0) and np.all(out["T"][0] == 1.0)
    one = sc.subset(np.arange(1))
    out = gpu_render(one, cams)
    ref = oracle.render(one, cams[0])
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="one splat")


def test_forward_into_a_caller_buffer(cuda_ok):
    """render_fwd(image=buf) composites the same image into buf (the end-to-end path
    renders straight into its staging buffer); a buffer of another size is refused on
    the host before anything is enqueued."""
    import torch
    sc, cams = scenes.config1()
    out = gpu_render(sc, cams)
    r = out["rast"]
    buf = torch.full_like(r.image, -1.0)
    r.clear_status()
    r.render_fwd(buf)
    assert r.read_status() == 0
    assert torch.equal(buf, r.image)
    with pytest.raises(ValueError):
        r.render_fwd(torch.empty(r.image.numel() - 1, device=r.image.device))


def test_forward_clears_the_backward_gradient_buffer(cuda_ok):
    """render_fwd clears grad2d (grad2d_clear) and the backward after it skips its own
    clearing; a second backward after the same forward clears it again.  All three
    give the gradients of a backward that clears grad2d itself, whatever grad2d held."""
    import torch
    from paper_2406_02720_b300 import hgs as H
    rng = np.random.default_rng(45)
    sc = scenes.scene_uniform(rng, 1500, [-1.5, -1.0, 2.5], [1.5, 1.0, 6.0], -3.2, 0.6, 1.5, 1)
    cams = [scenes.identity_camera(136, 88, 80.0)]
    out = gpu_render(sc, cams)
    r = out["rast"]
    dL = torch.from_numpy(np.asarray(scenes.upstream_grad(46, cams)[0], np.float32).reshape(-1)).cuda()

    def backward(clear_in_forward):
        r.grad2d.fill_(7.0)                       # stale contents
        r.clear_status()
        if clear_in_forward:
            r.render_fwd()
            r.rasterize_bwd(dL)
        else:
            r.render_fwd()
            r.grad2d.fill_(7.0)
            H.hgs_rasterize_bwd(r.proj_struct(), r.n, ctypes.c_void_p(r.ids.data_ptr()),
                                ctypes.c_void_p(r.ranges.data_ptr()), r.cams_host,
                                ctypes.c_void_p(r.cams_dev.data_ptr()), r.n_views, r.cfg,
                                ctypes.c_void_p(r.render_ws.data_ptr()), r.render_ws.numel(),
                                ctypes.c_void_p(r.final_T.data_ptr()), ctypes.c_void_p(r.n_contrib.data_ptr()),
                                ctypes.c_void_p(r.vis.data_ptr()), r.vis.numel(),
                                ctypes.c_void_p(dL.data_ptr()), ctypes.c_void_p(r.grad2d.data_ptr()), 0,
                                ctypes.c_void_p(r.status.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert r.read_status() == 0
        return r.grad2d.cpu().numpy().copy()

    ref = backward(False)
    got = backward(True)
    r.grad2d.fill_(7.0)
    r.rasterize_bwd(dL)                           # second backward after the same forward
    assert r.read_status() == 0
    again = r.grad2d.cpu().numpy()
    scale = np.abs(ref).max(axis=0) + 1e-30
    for g in (got, again):
        np.testing.assert_allclose(g / scale, ref / scale, rtol=0, atol=1e-6)
    assert np.count_nonzero(ref) > 1000
