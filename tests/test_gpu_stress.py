"""The stress workload at reduced splat count and full 1920x1080: 30% 100:1 disks
whose splitting planes are within 5 degrees of containing the ray (the
half-plane terms are then near-degenerate and take the FP64 path), against the
FP64 oracle; and its alpha2 := alpha1 copy, which must equal plain 3D-GS bit for
bit on the GPU."""
import numpy as np
import pytest

import oracle
from hgs_testutil import check_grads, compare_image, gpu_render, masked_upstream
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def test_grazing_disks_against_oracle(cuda_ok):
    sc, cams = scenes.config5(n=100_000)
    cam = cams[0]
    ref = oracle.render(sc, cam)
    pr = ref["proj"]
    # the scene really has near-degenerate half-planes: v / var_s small for many disks
    vis = pr["mode"] != oracle.CULLED
    ratio = pr["var_terms"][vis, 1] / np.maximum(pr["var_terms"][vis, 0], 1e-300)
    assert (ratio < 1e-3).sum() >= 20
    dL = masked_upstream(scenes.upstream_grad(105, cams), [ref])
    out = gpu_render(sc, cams, dL=dL)
    # the gathered FP64 list is the set of drawn splats with v < 1e-3 var_s (the GPU
    # decides in FP32, so only splats near the 1e-3 boundary may differ), and their
    # half-plane terms are the FP64 ones
    drawn = vis & (pr["tiles"] > 0)
    r_all = pr["var_terms"][:, 1] / np.maximum(pr["var_terms"][:, 0], 1e-300)
    want = np.flatnonzero(drawn & (pr["mode"] == oracle.NORMAL) & (r_all < 1e-3))
    got = out["fp64_fwd"].astype(np.int64)
    assert len(np.unique(got)) == len(got)
    diff = np.setxor1d(got, want)
    assert np.all(np.abs(r_all[diff] / 1e-3 - 1.0) < 1e-2), diff[:10]
    assert len(got) >= 20
    both = np.intersect1d(got, want)
    wp = out["rec"][0][both][:, 7:9].astype(np.float64)
    wr = pr["wp"][both]
    assert np.all(np.abs(wp - wr).max(1) <= 1e-5 * np.abs(wr).max(1)), np.abs(wp - wr).max()
    assert np.array_equal(out["keys"], ref["bins"]["keys"])
    assert np.array_equal(out["ids"], ref["bins"]["ids"])
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="grazing disks 100k")
    gref = oracle.render_bwd(sc, cam, dL[0], proj=pr, bins=ref["bins"])
    for k in ("means", "scales", "quats", "normals", "opac1", "opac2", "sh"):
        check_grads(out["grads"][k], gref[k], ref["touched"], label=f"grazing disks {k}", err=gref["err_" + k])


def test_equal_opacity_copy_is_plain_3dgs(cuda_ok):
    sc, cams = scenes.config5(n=40_000, equal_opacity=True)
    a = gpu_render(sc, cams)
    b = gpu_render(sc, cams, plain=True)
    assert np.array_equal(a["images"][0], b["images"][0])
    assert np.array_equal(a["T"][0], b["T"][0])
    assert np.array_equal(a["n_contrib"][0], b["n_contrib"][0])


def test_grazing_disks_with_mip(cuda_ok):
    """The same near-degenerate scene as Mip-Splatting-HGS: the opacity factor's
    adjoint also runs in the FP64 geometry adjoint of the gathered disks."""
    sc, cams = scenes.config5(n=60_000)
    cam = cams[0]
    ref = oracle.render(sc, cam, mip=True)
    pr = ref["proj"]
    dL = masked_upstream(scenes.upstream_grad(106, cams), [ref])
    out = gpu_render(sc, cams, dL=dL, mip=True)
    assert len(out["fp64_fwd"]) >= 10                   # the FP64 path is exercised
    compare_image(out["images"][0], out["T"][0], out["n_contrib"][0], ref, label="grazing disks mip")
    gref = oracle.render_bwd(sc, cam, dL[0], proj=pr, bins=ref["bins"], mip=True)
    for k in ("means", "scales", "quats", "normals", "opac1", "opac2", "sh"):
        check_grads(out["grads"][k], gref[k], ref["touched"], label=f"grazing disks mip {k}", err=gref["err_" + k])
