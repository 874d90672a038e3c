"""Pins of the oracle's per-half tile rectangle (rect_mode 1, the valid region of each
half of Sec. 3.4): a kept half's 3-sigma half-ellipsoid, projected by the affine map of
the EWA approximation, lies inside the rectangle and reaches its edges; with both halves
kept the rectangle is the closed-form bounding box of the projected 3-sigma ellipse (the
"tangent edges"); a half below the 1/255 floor is not splatted; and the rule is
symmetric under (n, alpha1, alpha2) -> (-n, alpha2, alpha1).  Tiles of 1x1 pixels make
the rectangle a pixel-level box."""
import numpy as np
import pytest

import oracle
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.filterwarnings("ignore")


def _scene(n, seed, alpha=(0.6, 0.6)):
    rng = np.random.default_rng(seed)
    sc = scenes.scene_uniform(rng, n, [-0.3, -0.3, 4.0], [0.3, 0.3, 6.0], -1.6, 0.5, 1.0, 0)
    sc.opac1[:] = alpha[0]
    sc.opac2[:] = alpha[1]
    return sc


CAM = scenes.identity_camera(1024, 1024, 900.0)


def _affine(sc, i):
    """mu-hat and M L of splat i in FP64 (identity camera: W = I)."""
    m = sc.means[i].astype(np.float64)
    q = sc.quats[i].astype(np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    L = R * sc.scales[i].astype(np.float64)[None, :]
    f = CAM.fx
    J = np.array([[f / m[2], 0, -f * m[0] / m[2] ** 2], [0, f / m[2], -f * m[1] / m[2] ** 2]])
    mu = np.array([f * m[0] / m[2] + CAM.cx, f * m[1] / m[2] + CAM.cy])
    return mu, J @ L, L


def _half_samples(L, n_vec, side, rng, k=4000):
    """Points L v of the 3-sigma half-ellipsoid on `side` of the plane (surface and cut disk)."""
    v = rng.standard_normal((k, 3))
    v = 3.0 * v / np.linalg.norm(v, axis=1, keepdims=True)
    pts = v @ L.T
    pts = pts[side * (pts @ n_vec) >= 0]
    # cut disk: directions in the plane n.(L v) = 0, i.e. v orthogonal to L^T n
    a = L.T @ n_vec
    basis = np.linalg.svd(a[None, :])[2][1:]          # two unit vectors orthogonal to a
    t = rng.uniform(0, 2 * np.pi, k)
    rad = 3.0 * np.sqrt(rng.uniform(0, 1, k))
    vd = rad[:, None] * (np.cos(t)[:, None] * basis[0] + np.sin(t)[:, None] * basis[1])
    return np.concatenate([pts, vd @ L.T])


def test_kept_half_projects_inside_its_rectangle_and_reaches_the_edges():
    rng = np.random.default_rng(5)
    for alpha, sides in (((0.6, 0.0), [1]), ((0.0, 0.6), [-1])):
        sc = _scene(60, 11, alpha)
        pr = oracle.project(sc, CAM, tile=(1, 1), lowpass=0.0, rect_mode=1)
        for i in range(sc.n):
            assert pr["tiles"][i] > 0
            x0, y0, x1, y1 = pr["rect"][i]
            mu, ML, L = _affine(sc, i)
            nv = sc.normals[i].astype(np.float64)
            pts = np.concatenate([_half_samples(L, nv, s, rng) for s in sides]) @ (ML @ np.linalg.inv(L)).T
            p = mu[None, :] + pts
            # pixel columns/rows of the samples, clamped to the grid as the rectangle is
            px = np.clip(np.floor(p[:, 0]), 0, 1023)
            py = np.clip(np.floor(p[:, 1]), 0, 1023)
            assert px.min() >= x0 - 1 and px.max() <= x1 and py.min() >= y0 - 1 and py.max() <= y1, i
            # tight: the sampled extremes come within 2 px of every edge inside the grid
            assert x0 == 0 or px.min() <= x0 + 2, i
            assert x1 == 1024 or px.max() >= x1 - 3, i
            assert y0 == 0 or py.min() <= y0 + 2, i
            assert y1 == 1024 or py.max() >= y1 - 3, i


def test_both_halves_kept_gives_the_ellipse_bounding_box():
    sc = _scene(200, 12, (0.6, 0.02))
    pr = oracle.project(sc, CAM, tile=(1, 1), rect_mode=1)
    a = pr["canon_abc"][:, 0].astype(np.float64)
    c = pr["canon_abc"][:, 2].astype(np.float64)
    mu = pr["canon_mu"].astype(np.float64)
    ex, ey = 3 * np.sqrt(a), 3 * np.sqrt(c)
    want = np.stack([np.floor(mu[:, 0] - ex), np.floor(mu[:, 1] - ey),
                     np.floor(mu[:, 0] + ex) + 1, np.floor(mu[:, 1] + ey) + 1], 1)
    want = np.clip(want, 0, 1024)                     # clamped to the grid of 1x1 tiles
    assert np.abs(pr["rect"] - want).max() <= 1
    # and it is never larger than the 3-sigma square of 3D-GS
    sq = oracle.project(sc, CAM, tile=(1, 1), rect_mode=0)
    assert np.all(pr["rect"][:, :2] >= sq["rect"][:, :2]) and np.all(pr["rect"][:, 2:] <= sq["rect"][:, 2:])


def test_transparent_halves_are_not_splatted():
    both = _scene(100, 13, (0.6, 0.6))
    one = _scene(100, 13, (0.6, 0.001))
    none = _scene(100, 13, (0.002, 0.003))
    rb = oracle.project(both, CAM, tile=(1, 1), rect_mode=1)
    r1 = oracle.project(one, CAM, tile=(1, 1), rect_mode=1)
    r0 = oracle.project(none, CAM, tile=(1, 1), rect_mode=1)
    assert np.all(r0["tiles"] == 0) and np.all(r0["mode"] == oracle.CULLED)
    assert np.all(r1["tiles"] <= rb["tiles"])
    assert np.mean(r1["tiles"] < rb["tiles"]) > 0.9          # oblique planes: the half is smaller
    # the 3-sigma square ignores the opacities
    s0 = oracle.project(none, CAM, tile=(1, 1), rect_mode=0)
    assert np.all(s0["tiles"] > 0)


def test_complement_symmetry_of_the_rectangle():
    a = _scene(150, 14, (0.6, 0.001))
    b = scenes.Scene(a.means, a.scales, a.quats, -a.normals, a.opac2.copy(), a.opac1.copy(), a.sh, a.sh_degree)
    ra = oracle.project(a, CAM, tile=(16, 16), rect_mode=1)
    rb = oracle.project(b, CAM, tile=(16, 16), rect_mode=1)
    assert np.array_equal(ra["rect"], rb["rect"]) and np.array_equal(ra["tiles"], rb["tiles"])
