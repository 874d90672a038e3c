"""More parity cases against the FP64 oracle: configuration 2 at full size (every
pixel and every gradient), the projection adjoint at each SH degree (each is its own
specialised kernel), near-degenerate half-planes seen from several views (the FP64
adjoint's atomics and the multi-view projection adjoint), and splats large enough to
cover every tile of a view."""
import numpy as np
import pytest

import oracle
from hgs_testutil import check_grads, compare_image, gpu_render, masked_upstream
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu

GRADS = ("means", "scales", "quats", "normals", "opac1", "opac2", "sh")


def _check_grads(out, gref, touched, label):
    for k in GRADS:
        check_grads(out["grads"][k], gref[k], touched, label=f"{label} {k}", err=gref["err_" + k])


def test_config2_full_parity(cuda_ok):
    """1280x720, 200k half-Gaussians, SH degree 3, upstream N(0,1): every pixel,
    every sorted pair and every parameter gradient."""
    sc, cams = scenes.config2()
    ref = oracle.render(sc, cams[0])
    dL = masked_upstream(scenes.upstream_grad(102, cams), [ref])
    out = gpu_render(sc, cams, dL=dL)
    assert np.array_equal(out["keys"], ref["bins"]["keys"])
    assert np.array_equal(out["ids"], ref["bins"]["ids"])
    assert np.array_equal(out["ranges"], ref["bins"]["ranges"])
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="config2")
    gref = oracle.render_bwd(sc, cams[0], dL[0], proj=ref["proj"], bins=ref["bins"])
    _check_grads(out, gref, ref["touched"], "config2")


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_gradients_each_sh_degree(cuda_ok, deg):
    rng = np.random.default_rng(60 + deg)
    sc = scenes.scene_uniform(rng, 500, [-1.3, -0.8, 2.5], [1.3, 0.8, 6], -3.3, 0.5, 1.5, deg)
    cams = [scenes.identity_camera(128, 80, 80.0, bg=(0.2, 0.1, 0.3))]
    ref = oracle.render(sc, cams[0])
    dL = masked_upstream(scenes.upstream_grad(70 + deg, cams), [ref])
    out = gpu_render(sc, cams, dL=dL)
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label=f"SH degree {deg}")
    gref = oracle.render_bwd(sc, cams[0], dL[0], proj=ref["proj"], bins=ref["bins"])
    _check_grads(out, gref, ref["touched"], f"SH degree {deg}")


def test_grazing_disks_from_two_views(cuda_ok):
    """Near-degenerate planes in a two-view step: the per-view FP64 lists, their atomic
    adds into one splat's gradient, and the multi-view projection adjoint."""
    sc, cams0 = scenes.config5(n=60_000)
    eye = np.array([1.0, 0.5, -12.0])
    small = [cams0[0], scenes.look_at_camera(eye, [0.0, 0.0, 0.0], [0.0, 1.0, 0.0], 960, 540, 750.0)]
    refs = [oracle.render(sc, c) for c in small]
    r0 = refs[0]["proj"]
    vis = r0["mode"] == oracle.NORMAL
    ratio = r0["var_terms"][vis, 1] / np.maximum(r0["var_terms"][vis, 0], 1e-300)
    assert (ratio < 1e-3).sum() >= 20
    dL = masked_upstream(scenes.upstream_grad(80, small), refs)
    out = gpu_render(sc, small, dL=dL)
    for v in range(2):
        compare_image(out["images"][v], out["T"][v], out["n_contrib"][v], refs[v], label=f"grazing view {v}")
    tot = None
    for c, d, r in zip(small, dL, refs):
        g = oracle.render_bwd(sc, c, d, proj=r["proj"], bins=r["bins"])
        tot = g if tot is None else {k: tot[k] + g[k] for k in tot}
    _check_grads(out, tot, refs[0]["touched"] | refs[1]["touched"], "grazing two views")


def test_splats_covering_every_tile(cuda_ok):
    """A few splats near the camera cover all 920 tiles of a 640x360 view, so one warp
    of the pair emission expands thousands of pairs and every tile list is long."""
    rng = np.random.default_rng(90)
    sc = scenes.scene_uniform(rng, 3000, [-2.0, -1.2, 3.0], [2.0, 1.2, 8.0], -3.0, 0.6, 1.5, 1)
    big = np.arange(4)
    sc.means[big] = [[0.0, 0.0, 2.5], [0.3, -0.2, 3.0], [-0.4, 0.1, 3.5], [0.1, 0.3, 4.0]]
    sc.scales[big] = 1.5
    sc.opac1[big] = 0.3
    sc.opac2[big] = 0.02
    cams = [scenes.identity_camera(640, 360, 400.0, bg=(0.0, 0.0, 0.0))]
    ref = oracle.render(sc, cams[0])
    assert (ref["proj"]["tiles"][big] == 920).all()
    dL = masked_upstream(scenes.upstream_grad(91, cams), [ref])
    out = gpu_render(sc, cams, dL=dL)
    assert np.array_equal(out["keys"], ref["bins"]["keys"])
    assert np.array_equal(out["ids"], ref["bins"]["ids"])
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="covering")
    gref = oracle.render_bwd(sc, cams[0], dL[0], proj=ref["proj"], bins=ref["bins"])
    _check_grads(out, gref, ref["touched"], "covering")
