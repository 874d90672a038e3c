"""Pins of the oracle's per-half tile rectangle (rect_mode 1, the valid region of each
half of Sec. 3.4): a kept half's 3-sigma half-ellipsoid, projected by the affine map of
the EWA approximation, lies inside the rectangle and reaches its edges; with both halves
kept the rectangle is the closed-form bounding box of the projected 3-sigma ellipse (the
"tangent edges"); a half below the 1/255 floor is not splatted; and the rule is
symmetric under (n, alpha1, alpha2) -> (-n, alpha2, alpha1).  Tiles of 1x1 pixels make
the rectangle a pixel-level box.

rect_mode 2 takes the splitting edge from Algorithm 1 (Suppl. B.1).  Its FP64 form is
pinned against the block-inverse identity (the in-plane block of the flattened
covariance is the inverse of the plane's block of the precision matrix), the normal
as an eigenvector with variance min(a', c') / 100, the axis-aligned special case, and
the cut ellipse lying on the flattened ellipsoid's 3-sigma surface; the oracle's
binary32 rectangles are pinned against extents recomputed from the FP64 algorithm, and
they contain the exact cut-ellipse rectangles of rect_mode 1."""
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


def _random_cov(rng):
    A = rng.standard_normal((3, 3)) * np.array([1.0, 0.4, 0.1])[None, :]
    return A @ A.T + 1e-6 * np.eye(3)


def _plane_basis(n):
    """Two orthonormal vectors orthogonal to n, from an SVD (not Algorithm 1's choice)."""
    return np.linalg.svd(n[None, :])[2][1:].T          # 3 x 2


def test_alg1_in_plane_block_is_the_conditional_covariance():
    rng = np.random.default_rng(40)
    for _ in range(200):
        S = _random_cov(rng)
        n = rng.standard_normal(3)
        sig = oracle.alg1_flat_cov(S, n)
        W = _plane_basis(n)
        want = np.linalg.inv(W.T @ np.linalg.inv(S) @ W)
        np.testing.assert_allclose(W.T @ sig @ W, want, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(sig, sig.T, atol=1e-14)


def test_alg1_normal_axis_is_an_eigenvector_with_a_hundredth_of_the_smaller_variance():
    rng = np.random.default_rng(41)
    for _ in range(200):
        S = _random_cov(rng)
        n = rng.standard_normal(3)
        h = n / np.linalg.norm(n)
        sig = oracle.alg1_flat_cov(S, n)
        # no cross term between the plane and the normal direction
        np.testing.assert_allclose(sig @ h - (h @ sig @ h) * h, 0.0, atol=1e-12 * np.abs(sig).max())
        # the paper's in-plane axes: v1 = (n_y, -n_x, 0) / |.|, v2 = n x v1
        v1 = np.array([h[1], -h[0], 0.0]) / np.hypot(h[0], h[1])
        v2 = np.cross(h, v1)
        cond = np.linalg.inv(_plane_basis(n).T @ np.linalg.inv(S) @ _plane_basis(n))
        W = _plane_basis(n)
        C = W @ cond @ W.T                              # conditional covariance, as a 3x3 map
        want = min(v1 @ C @ v1, v2 @ C @ v2) / 100.0
        assert abs(h @ sig @ h - want) <= 1e-10 * want
        assert np.linalg.eigvalsh(sig).min() > 0.0


def test_alg1_axis_aligned_normal():
    """n along z: v1 = x, v2 = y, and the in-plane block is the Schur complement of z."""
    rng = np.random.default_rng(42)
    S = _random_cov(rng)
    sig = oracle.alg1_flat_cov(S, np.array([0.0, 0.0, 2.5]))
    schur = S[:2, :2] - np.outer(S[:2, 2], S[2, :2]) / S[2, 2]
    np.testing.assert_allclose(sig[:2, :2], schur, rtol=1e-12)
    np.testing.assert_allclose(sig[:2, 2], 0.0, atol=1e-15)
    assert sig[2, 2] == pytest.approx(min(schur[0, 0], schur[1, 1]) / 100.0, rel=1e-12)


def test_alg1_cut_ellipse_lies_on_the_flattened_3sigma_surface():
    rng = np.random.default_rng(43)
    for _ in range(50):
        S = _random_cov(rng)
        n = rng.standard_normal(3)
        sig = oracle.alg1_flat_cov(S, n)
        W = _plane_basis(n)
        # points of the plane on the original 3-sigma surface: x = W y, x^T S^-1 x = 9
        Q = W.T @ np.linalg.inv(S) @ W
        t = rng.uniform(0, 2 * np.pi, 64)
        y = np.stack([np.cos(t), np.sin(t)], 1)
        y = 3.0 * y / np.sqrt(np.einsum("ki,ij,kj->k", y, Q, y))[:, None]
        x = y @ W.T
        d2 = np.einsum("ki,ij,kj->k", x, np.linalg.inv(sig), x)
        np.testing.assert_allclose(d2, 9.0, rtol=1e-8)


def _alg1_rect_fp64(sc, i, side_keep, lp):
    """Pixel rectangle of splat i under rect_mode 2 recomputed in FP64 (1x1 tiles):
    per kept half and direction, the whole ellipse's extent where the half's outer
    edge faces that way (sign of k = J Sigma n^), else the extent of the projected
    flattened covariance of Algorithm 1."""
    mu, ML, L = _affine(sc, i)
    J = ML @ np.linalg.inv(L)
    S = L @ L.T
    n = sc.normals[i].astype(np.float64)
    h = n / np.linalg.norm(n)
    k = J @ S @ h
    full = np.diag(J @ S @ J.T)
    flat = np.diag(J @ oracle.alg1_flat_cov(S, n) @ J.T)
    ext = {}
    for axis, (kk, f, c) in enumerate(zip(k, full, flat)):
        plus = minus = 0.0
        for side, keep in ((1, side_keep[0]), (-1, side_keep[1])):
            if not keep:
                continue
            plus = max(plus, f if side * kk >= 0 else c)
            minus = max(minus, f if side * kk <= 0 else c)
        ext[axis] = (3 * np.sqrt(minus + lp), 3 * np.sqrt(plus + lp))
    lo = [np.floor(mu[a] - ext[a][0]) for a in (0, 1)]
    hi = [np.floor(mu[a] + ext[a][1]) + 1 for a in (0, 1)]
    return np.clip(np.array([lo[0], lo[1], hi[0], hi[1]]), 0, 1024)


def test_rect_mode2_matches_fp64_algorithm1():
    for alpha in ((0.6, 0.0), (0.0, 0.6), (0.6, 0.6)):
        sc = _scene(120, 44, alpha)
        pr = oracle.project(sc, CAM, tile=(1, 1), lowpass=0.3, rect_mode=2)
        keep = (alpha[0] >= 1 / 255, alpha[1] >= 1 / 255)
        for i in range(sc.n):
            want = _alg1_rect_fp64(sc, i, keep, 0.3)
            assert np.abs(pr["rect"][i] - want).max() <= 1, (alpha, i, pr["rect"][i], want)


def test_rect_mode2_contains_the_cut_ellipse_rectangle():
    """The flattened ellipsoid holds the cut ellipse, so its rectangles hold rect_mode 1's,
    and they stay below the 3-sigma square's pair count."""
    for alpha in ((0.6, 0.001), (0.001, 0.6)):
        sc = _scene(300, 45, alpha)
        r1 = oracle.project(sc, CAM, tile=(1, 1), rect_mode=1)
        r2 = oracle.project(sc, CAM, tile=(1, 1), rect_mode=2)
        r0 = oracle.project(sc, CAM, tile=(1, 1), rect_mode=0)
        assert np.all(r2["rect"][:, :2] <= r1["rect"][:, :2]) and np.all(r2["rect"][:, 2:] >= r1["rect"][:, 2:])
        assert r2["tiles"].sum() < r0["tiles"].sum()
        assert r2["tiles"].sum() <= 1.05 * r1["tiles"].sum()


def test_rect_mode2_complement_symmetry():
    a = _scene(150, 46, (0.6, 0.001))
    b = scenes.Scene(a.means, a.scales, a.quats, -a.normals, a.opac2.copy(), a.opac1.copy(), a.sh, a.sh_degree)
    ra = oracle.project(a, CAM, tile=(16, 16), rect_mode=2)
    rb = oracle.project(b, CAM, tile=(16, 16), rect_mode=2)
    assert np.array_equal(ra["rect"], rb["rect"]) and np.array_equal(ra["tiles"], rb["tiles"])
