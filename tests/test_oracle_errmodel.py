"""Pins of the oracle's FP32 error model (reading B15), which decides the threshold
decisions a binary32 implementation cannot be expected to reproduce and bounds
the error of a binary32 evaluation of the gradients.  Each check ties the model
to something outside it: closed forms of the perturbation basis, an actual
binary32 evaluation of hat Sigma, a decision that really flips, and the
Jacobian of the forward projection by finite differences."""
import numpy as np
import pytest

import oracle
from paper_2406_02720_b300 import scenes

U32 = 2.0 ** -24
T_Z, RC, SCALE, QUAT, NORMAL = 2, slice(3, 12), slice(12, 15), slice(15, 19), slice(19, 22)


def _one(mean, scale, quat, normal, a1=0.5, a2=0.5):
    f32 = lambda x: np.asarray(x, np.float32).reshape(1, -1)     # noqa: E731
    return scenes.Scene(f32(mean), f32(scale), f32(quat), f32(normal), np.float32([a1]), np.float32([a2]),
                        np.zeros((1, 1, 3), np.float32), 0)


def test_error_basis_closed_form_on_axis():
    """Isotropic splat on the optical axis, no low-pass: conic = (z / (f s))^2 I and
    w' = (z/f)(n1, n2) / (s |n3| sqrt 2).  Per unit relative perturbation: depth
    z -> (2A, 0, 2C, w'x, w'y); scale s_k (k = x, y) -> -2 of the matching conic
    entry; the scale along the ray and the unit quaternion's zero entries -> 0."""
    f, z, s = 200.0, 3.0, 0.05
    n = np.array([0.3, -0.4, 0.866])
    sc = _one([0.0, 0.0, z], [s, s, s], [1.0, 0.0, 0.0, 0.0], n)
    cam = scenes.identity_camera(64, 64, f)
    pr = oracle.project(sc, cam, lowpass=0.0, errmat=False)
    E, V = oracle.error_basis(sc, cam, pr["mode"], lowpass=0.0, vectors=True)
    V = V[0]
    z, s = float(np.float32(z)), float(np.float32(s))      # the scene holds binary32 values
    n = np.float32(n).astype(np.float64)
    A = (z / (f * s)) ** 2
    nh = n / np.linalg.norm(n)
    wp = (z / f) * nh[:2] / (s * abs(nh[2]) * np.sqrt(2.0))
    np.testing.assert_allclose(pr["conic"][0], [A, 0.0, A], rtol=1e-12)
    np.testing.assert_allclose(pr["wp"][0], wp, rtol=1e-9)
    np.testing.assert_allclose(V[T_Z], [2 * A, 0.0, 2 * A, wp[0], wp[1]], rtol=1e-6, atol=1e-9 * A)
    sv = V[SCALE]
    np.testing.assert_allclose(sv[0, [0, 1, 2]], [-2 * A, 0.0, 0.0], rtol=1e-6, atol=1e-9 * A)
    np.testing.assert_allclose(sv[1, [0, 1, 2]], [0.0, 0.0, -2 * A], rtol=1e-6, atol=1e-9 * A)
    np.testing.assert_allclose(sv[2, [0, 1, 2]], 0.0, atol=1e-9 * A)
    np.testing.assert_allclose(V[QUAT][1:], 0.0, atol=0)           # exact zeros stay exact
    np.testing.assert_allclose(V[QUAT][0], 0.0, atol=1e-9 * A)      # scaling q changes nothing
    # E is the sum of the outer products
    full = np.zeros((5, 5))
    k = 0
    for a in range(5):
        for b in range(a, 5):
            full[a, b] = full[b, a] = E[0, k]
            k += 1
    np.testing.assert_allclose(full, V.T @ V, rtol=1e-12, atol=1e-30)


def _binary32_conic(sc, cam, i, lp):
    """hat Sigma^-1 of splat i with L = R diag(s), M = J W and P = M L each held in
    binary32 (every product that carries the splat's shape into screen space rounded
    once), and hat Sigma = P P^T + l I, its determinant and inverse formed exactly
    (FP64) from that P: a binary32 evaluation of the shape in which nothing cancels
    after the rounding, the property of the design's cancellation-free determinant."""
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)      # noqa: E731
    q = sc.quats[i].astype(np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    L = f32(R * sc.scales[i].astype(np.float64)[None, :])
    V = np.asarray(cam.viewmat, np.float64)
    t = V[:, :3] @ sc.means[i].astype(np.float64) + V[:, 3]
    J = np.array([[cam.fx / t[2], 0.0, -cam.fx * t[0] / t[2] ** 2], [0.0, cam.fy / t[2], -cam.fy * t[1] / t[2] ** 2]])
    M = f32(J @ V[:, :3])
    P = f32(M @ L)
    S = P @ P.T + lp * np.eye(2)
    Qm = np.linalg.inv(S)
    return np.array([Qm[0, 0], Qm[0, 1], Qm[1, 1]])


def test_shape_band_covers_a_binary32_evaluation_of_hat_sigma():
    """The exponent of a binary32 evaluation of the shape (_binary32_conic) at pixel
    offsets inside the 3-sigma ellipse differs from the FP64 one by no more than the
    model's shape term 8 u sqrt(g^T E g) (doubled), for every sampled splat and offset,
    thin splats included; and for thin splats the model's term is not vacuous (it is
    within 10^3 of the observed difference)."""
    rng = np.random.default_rng(7)
    sc = scenes.scene_uniform(rng, 2000, [-1.5, -1.0, 2.0], [1.5, 1.0, 6.0], -3.5, 1.2, 1.0, 0)
    cam = scenes.identity_camera(200, 150, 150.0)
    lp = float(np.float32(0.3))
    pr = oracle.project(sc, cam)
    live = np.flatnonzero(pr["mode"] == oracle.NORMAL)
    worst, thin, ratios = 0.0, 0, []
    for i in live:
        Q = pr["conic"][i]
        Q32 = _binary32_conic(sc, cam, i, lp)
        S = np.linalg.inv([[Q[0], Q[1]], [Q[1], Q[2]]])
        ev = np.linalg.eigvalsh(S)
        is_thin = ev[1] / ev[0] > 30
        thin += is_thin
        Lc = np.linalg.cholesky(S)
        E = np.zeros((5, 5))
        k = 0
        for a in range(5):
            for b in range(a, 5):
                E[a, b] = E[b, a] = pr["errmat"][i, k]
                k += 1
        for _ in range(6):
            d = Lc @ rng.uniform(-3, 3, 2)
            g = np.array([-0.5 * d[0] ** 2, -d[0] * d[1], -0.5 * d[1] ** 2, 0.0, 0.0])
            band = 2.0 * 8.0 * U32 * np.sqrt(max(g @ E @ g, 0.0))
            dq = Q32 - Q
            diff = abs(0.5 * (dq[0] * d[0] ** 2 + 2 * dq[1] * d[0] * d[1] + dq[2] * d[1] ** 2))
            worst = max(worst, diff / band)
            if is_thin and diff > 0:
                ratios.append(band / diff)
    assert thin > 20                      # thin splats are part of the sample
    assert worst <= 1.0, worst
    assert np.median(ratios) < 1e3


def test_flip_bound_covers_a_flipped_floor_decision():
    """A splat whose weight at one pixel sits at 1/255 (1 + 1e-9): that decision is
    marked (margin <= 1), and moving the weight to 1/255 (1 - 1e-9), which flips it,
    changes the pixel by no more than the oracle's flip bounds."""
    cam = scenes.identity_camera(32, 32, 40.0, bg=(0.1, 0.2, 0.3))
    s = 0.2
    mean, back = [0.0, 0.0, 2.0], [0.05, -0.03, 3.0]
    px, py = 16.5 + 3.0, 16.5       # the pixel centre examined
    sc = _one(mean, [s, s, s], [1.0, 0.0, 0.0, 0.0], [0.0, 0.0, 1.0])
    G, P, _ = oracle.eval_splat(sc.means[0], sc.scales[0], sc.quats[0], sc.normals[0], cam, [px], [py])

    def scene(rel):
        alpha = np.float32((1.0 / 255.0) * (1.0 + rel) / G[0])
        two = scenes.Scene(np.float32([mean, back]), np.float32([[s, s, s], [0.4, 0.4, 0.4]]),
                           np.float32([[1, 0, 0, 0], [1, 0, 0, 0]]), np.float32([[0, 0, 1], [0, 0, 1]]),
                           np.float32([alpha, 0.8]), np.float32([alpha, 0.8]),
                           np.float32([[[1.2, -1.0, 0.4]], [[-1.0, 0.9, -0.5]]]), 0)
        return two, alpha

    above, a_hi = scene(1e-6)
    below, a_lo = scene(-1e-6)
    assert a_hi != a_lo                                   # the binary32 opacities differ
    r1, r2 = oracle.render(above, cam), oracle.render(below, cam)
    j, i = int(py), int(px)
    assert r1["margin_a"][j, i] <= 1.0 < r2["margin_a"].max()
    di = np.abs(r1["image"][:, j, i] - r2["image"][:, j, i]).max()
    dT = abs(r1["T"][j, i] - r2["T"][j, i])
    assert di > 1e-4                                      # the flip is visible ...
    assert di <= r1["flip_img"][j, i] and dT <= r1["flip_T"][j, i]     # ... and bounded
    assert r1["touched"][0] and not r1["touched"][1]


def test_parameter_error_bound_is_abs_jacobian_transpose():
    """param_error_bound(x) = |J|^T x per splat, J the Jacobian of the screen-space
    quantities (centre, conic, w', opacities, colour) w.r.t. the parameters, here by
    central differences of the forward projection."""
    rng = np.random.default_rng(11)
    sc = scenes.scene_uniform(rng, 6, [-0.5, -0.5, 2.5], [0.5, 0.5, 4.0], -2.5, 0.4, 1.0, 1)
    sc = scenes.Scene(*(np.asarray(a, np.float64) for a in sc.arrays()), sc.sh_degree)
    cam = scenes.identity_camera(96, 96, 90.0)
    pr = oracle.project(sc, cam, errmat=False)
    assert np.all(pr["mode"] == oracle.NORMAL)
    x = rng.uniform(0.5, 2.0, (sc.n, 12))
    bound = oracle.param_error_bound(sc, cam, pr["mode"], np.zeros((sc.n, 12)), x)

    def screen(s):
        p = oracle.project(s, cam, errmat=False)
        return np.concatenate([p["mu2"], p["conic"], p["wp"], p["opac1"][:, None], p["opac2"][:, None], p["rgb"]], 1)

    for name in ("means", "scales", "quats", "normals"):
        arr = getattr(sc, name)
        want = np.zeros_like(arr)
        for k in range(arr.shape[1]):
            h = 1e-6 * np.maximum(np.abs(arr[:, k]), 1e-3)
            plus, minus = [scenes.Scene(*(a.copy() for a in sc.arrays()), sc.sh_degree) for _ in range(2)]
            getattr(plus, name)[:, k] += h
            getattr(minus, name)[:, k] -= h
            J = (screen(plus) - screen(minus)) / (2 * h[:, None])
            want[:, k] = np.sum(np.abs(J) * x, 1)
        np.testing.assert_allclose(bound[name], want, rtol=2e-5, atol=1e-9 * np.abs(want).max())


def _f32_pair_weight(sc, cam, i, px, py, lp, wp64, fp64_w):
    """A binary32 evaluation of splat i's pair weight at pixel centres (px, py), in the
    formulation the band is written for: L, M and P = M L rounded to binary32; hat Sigma's
    entries, its cancellation-free determinant |p0 x p1|^2 + l(|p0|^2 + |p1|^2) + l^2 and
    the conic's Cholesky factor in binary32; the half-plane terms likewise (FP64 w' where
    the plane nearly contains the ray); the pixel offset from tile-local binary32 numbers
    around an accurate centre; the exponent |U d|^2, exp and erfc in binary32."""
    f = np.float32
    q = sc.quats[i].astype(f)
    qn = np.sqrt(f(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]))
    w, x, y, z = (q / qn).astype(f)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]], f)
    L = (R * sc.scales[i].astype(f)[None, :]).astype(f)
    V = np.asarray(cam.viewmat, f)
    t = (V[:, :3] @ sc.means[i].astype(f) + V[:, 3]).astype(f)
    fx, fy = f(cam.fx), f(cam.fy)
    J = np.array([[fx / t[2], 0, -(fx * (t[0] / t[2])) / t[2]], [0, fy / t[2], -(fy * (t[1] / t[2])) / t[2]]], f)
    M = (J @ V[:, :3]).astype(f)
    P = (M @ L).astype(f)
    lpf = f(lp)
    a = f(P[0] @ P[0] + lpf)
    b = f(P[0] @ P[1])
    c = f(P[1] @ P[1] + lpf)
    cr = np.cross(P[0], P[1]).astype(f)
    det = f(cr @ cr + lpf * (P[0] @ P[0] + P[1] @ P[1]) + lpf * lpf)
    u11, u12, u22 = np.sqrt(c / det).astype(f), f(-b / np.sqrt(f(c * det))), f(1 / np.sqrt(c))
    if fp64_w:
        wpx, wpy = f(wp64[0]), f(wp64[1])
    else:
        nrm = sc.normals[i].astype(f)
        nh = (nrm / np.sqrt(f(nrm @ nrm))).astype(f)
        uu = (L.T @ nh).astype(f)
        k0, k1 = f(P[0] @ uu), f(P[1] @ uu)
        up0, up1 = np.cross(uu, P[0]).astype(f), np.cross(uu, P[1]).astype(f)
        trip = f(uu @ cr)
        v = f((trip * trip + lpf * (up0 @ up0 + up1 @ up1) + lpf * lpf * (uu @ uu)) / det)
        sv = f(1 / np.sqrt(f(2 * v)))
        wpx, wpy = f((c * k0 - b * k1) / det * sv), f((a * k1 - b * k0) / det * sv)
    mu = oracle.project(sc.subset([i]), cam, errmat=False)["mu2"][0]
    ox, oy = np.floor(px / 16) * 16, np.floor(py / 16) * 16
    mx, my = (mu[0] - ox).astype(f), (mu[1] - oy).astype(f)
    dx, dy = (px - ox).astype(f) - mx, (py - oy).astype(f) - my
    fma = lambda p_, q_, r_: f(np.float64(p_) * np.float64(q_) + np.float64(r_))     # noqa: E731
    s1 = fma(u11, dx, f(u12 * dy))
    s2 = f(u22 * dy)
    G = np.exp(f(-0.5) * fma(s1, s1, f(s2 * s2))).astype(f)
    zz = fma(wpx, dx, f(wpy * dy))
    from scipy.special import erfc
    Pf = f(0.5 * erfc(-np.float64(zz)))
    o1, o2 = f(sc.opac1[i]), f(sc.opac2[i])
    return f(fma(f(o1 - o2), Pf, o2) * G)


def test_band_covers_a_binary32_evaluation_of_the_pair_weight():
    """For every sampled (splat, pixel) pair inside the 3-sigma ellipse, thin splats and
    planes close to the ray included, |ln a32 - ln a| of the binary32 evaluation above
    stays within the oracle's band, and the band is not vacuous (its median is under
    100 times the observed difference)."""
    rng = np.random.default_rng(12)
    sc = scenes.scene_uniform(rng, 400, [-1.2, -0.9, 2.5], [1.2, 0.9, 5.5], -3.2, 1.1, 1.0, 0)
    cam = scenes.identity_camera(192, 144, 160.0)
    lp = float(np.float32(0.3))
    pr = oracle.project(sc, cam)
    vr = pr["var_terms"][:, 1] / np.maximum(pr["var_terms"][:, 0], 1e-300)
    ids, pxs, pys, worst, ratios = [], [], [], 0.0, []
    for i in np.flatnonzero(pr["mode"] == oracle.NORMAL):
        Q = pr["conic"][i]
        S = np.linalg.inv([[Q[0], Q[1]], [Q[1], Q[2]]])
        off = np.linalg.cholesky(S) @ rng.uniform(-2.5, 2.5, (2, 8))
        px = np.floor(pr["mu2"][i, 0] + off[0]) + 0.5
        py = np.floor(pr["mu2"][i, 1] + off[1]) + 0.5
        band, a64 = oracle.pair_bands(pr, np.full(px.size, i), px, py)
        a32 = _f32_pair_weight(sc, cam, i, px, py, lp, pr["wp"][i], vr[i] < 1e-3)
        ok = (band > 0) & (a64 > 1e-7) & (a32 > 0)
        d = np.abs(np.log(a32[ok].astype(np.float64)) - np.log(a64[ok]))
        if d.size:
            worst = max(worst, float((d / band[ok]).max()))
            ratios.extend(band[ok][d > 0] / d[d > 0])
    assert len(ratios) > 1000
    assert worst <= 1.0, worst
    assert np.median(ratios) < 100.0, np.median(ratios)
