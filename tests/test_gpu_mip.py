"""Mip-Splatting-HGS mode (hgs_config.mip) on the GPU against the oracle's mip mode:
the compensated opacities of the records, images and parameter gradients (one view
and two views, so both projection kernels run), and the l = 0 reduction to the plain
low-pass-free kernel (bitwise images)."""
import numpy as np
import pytest

import oracle
from hgs_testutil import check_grads, compare_image, gpu_render, masked_upstream
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu

FIELDS = ("means", "scales", "quats", "normals", "opac1", "opac2", "sh")


def _scene(seed, n=900):
    rng = np.random.default_rng(seed)
    # small footprints (0.3 - 3 px), where the 2D filter's factor is far from 1
    sc = scenes.scene_uniform(rng, n, [-1.3, -0.8, 2.5], [1.3, 0.8, 6], -4.2, 0.6, 1.5, 2)
    cams = [scenes.identity_camera(160, 96, 90.0, 80.0, 48.0, bg=(0.2, 0.3, 0.1))]
    return sc, cams


def test_mip_records_images_and_gradients(cuda_ok):
    sc, cams = _scene(41)
    ref = oracle.render(sc, cams[0], mip=True)
    dL = masked_upstream(scenes.upstream_grad(42, cams), [ref])
    out = gpu_render(sc, cams, dL=dL, mip=True)
    pr = ref["proj"]
    live = pr["mode"] != oracle.CULLED
    comp = pr["comp"][live]
    assert comp.min() < 0.5 and comp.max() < 1.0          # the factor matters here
    rec = out["rec"][0][live]
    for col, key in ((9, "opac1"), (10, "opac2")):
        np.testing.assert_allclose(rec[:, col], pr[key][live], rtol=2e-5, atol=1e-7)
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="mip")
    gref = oracle.render_bwd(sc, cams[0], dL[0], proj=ref["proj"], bins=ref["bins"], mip=True)
    for k in FIELDS:
        check_grads(out["grads"][k], gref[k], ref["touched"], label=f"mip {k}", err=gref["err_" + k])


def test_mip_two_views_gradients(cuda_ok):
    sc, cams = _scene(43, n=600)
    vm = np.asarray(cams[0].viewmat, np.float32).copy()
    vm[0, 3] += 0.15
    cams.append(scenes.Camera(vm, 80.0, 80.0, 64.0, 40.0, 128, 80, bg=(0.0, 0.0, 0.0)))
    refs = [oracle.render(sc, c, mip=True) for c in cams]
    dL = masked_upstream(scenes.upstream_grad(44, cams), refs)
    out = gpu_render(sc, cams, dL=dL, mip=True)
    total = None
    for v, c in enumerate(cams):
        compare_image(out["images"][v], out["T"][v], out["n_contrib"][v], refs[v], label=f"mip view {v}")
        g = oracle.render_bwd(sc, c, dL[v], proj=refs[v]["proj"], bins=refs[v]["bins"], mip=True)
        total = g if total is None else {k: total[k] + g[k] for k in total}
    touched = refs[0]["touched"] | refs[1]["touched"]
    for k in FIELDS:
        check_grads(out["grads"][k], total[k], touched, label=f"mip two views {k}", err=total["err_" + k])


def test_mip_without_lowpass_is_bitwise_the_plain_path(cuda_ok):
    sc, cams = _scene(45, n=500)
    a = gpu_render(sc, cams, lowpass=0.0, mip=True)
    b = gpu_render(sc, cams, lowpass=0.0, mip=False)
    assert np.array_equal(a["rec"], b["rec"])
    assert np.array_equal(a["images"][0], b["images"][0])


def test_mip_with_per_half_rectangles(cuda_ok):
    """mip with rect_mode 1: binning bit-exact against the oracle (its per-half test
    uses the unscaled opacities on both sides), images and gradients within tolerance."""
    rng = np.random.default_rng(47)
    sc = scenes.scene_uniform(rng, 1500, [-1.6, -1.0, 2.0], [1.6, 1.0, 7.0], -3.6, 0.6, 1.2, 1)
    k = rng.random(sc.n)
    sc.opac2[k < 0.3] = 0.002                          # one half below 1/255
    cams = [scenes.identity_camera(160, 96, 110.0, bg=(0.1, 0.1, 0.2))]
    ref = oracle.render(sc, cams[0], rect_mode=1, mip=True)
    dL = masked_upstream(scenes.upstream_grad(48, cams), [ref])
    out = gpu_render(sc, cams, dL=dL, rect_mode=1, mip=True)
    assert np.array_equal(out["keys"], ref["bins"]["keys"]) and np.array_equal(out["ids"], ref["bins"]["ids"])
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="mip rect_mode 1")
    gref = oracle.render_bwd(sc, cams[0], dL[0], proj=ref["proj"], bins=ref["bins"], mip=True)
    for f in FIELDS:
        check_grads(out["grads"][f], gref[f], ref["touched"], label=f"mip rect_mode 1 {f}", err=gref["err_" + f])
