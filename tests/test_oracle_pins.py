"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
not by the oracle itself (CPU only).

* Eq. 7-8 / Suppl. A.1: the half-Gaussian integral along the (affine) ray,
  done by numerical quadrature, against the oracle's hat G and P.
* The 3D-GS low-pass read as the EWA screen filter of the half footprint:
  a 2-D Gauss-Hermite convolution of the unfiltered P*hat G.
* Closed-form single splats (on the optical axis, isotropic scale).
* Sec. 3.2: alpha1 = alpha2 is exactly 3D-GS; the complementary half is the
  same kernel with -n.
* Real SH against scipy.special.sph_harm_y.
* Binning against brute force (tile/interval intersection, Python sort).
* Compositing identity: with white splats over black, image = 1 - T exactly.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special
from scipy.spatial.transform import Rotation

import oracle
from paper_2406_02720_b300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


class Cam:
    def __init__(self, viewmat, f, W, H, cx=None, cy=None, bg=(0, 0, 0), near=0.2):
        self.viewmat = np.asarray(viewmat, np.float64)
        self.fx = self.fy = float(f)
        self.cx = W / 2 if cx is None else cx
        self.cy = H / 2 if cy is None else cy
        self.width, self.height = W, H
        self.bg, self.near = bg, near


class Sc:
    def __init__(self, means, scales, quats, normals, o1, o2, sh, deg):
        self.means = np.asarray(means, np.float64).reshape(-1, 3)
        self.scales = np.asarray(scales, np.float64).reshape(-1, 3)
        self.quats = np.asarray(quats, np.float64).reshape(-1, 4)
        self.normals = np.asarray(normals, np.float64).reshape(-1, 3)
        self.opac1 = np.asarray(o1, np.float64).reshape(-1)
        self.opac2 = np.asarray(o2, np.float64).reshape(-1)
        n = self.means.shape[0]
        self.sh = np.asarray(sh, np.float64).reshape(n, -1, 3)
        self.sh_degree = deg


def _random_view(rng):
    """A random rotation and a translation that keeps the origin region in front."""
    rot = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
    vm = np.zeros((3, 4))
    vm[:, :3] = rot
    vm[:, 3] = [0.1, -0.2, 6.0]
    return vm


def _pixel_map(vm, f, cx, cy):
    def pi(x):
        xc = vm[:, :3] @ x + vm[:, 3]
        return np.array([f * xc[0] / xc[2] + cx, f * xc[1] / xc[2] + cy])
    return pi


def _jacobian_complex_step(fun, x, h=1e-30):
    """d fun / dx by the complex-step method (exact to rounding for analytic maps)."""
    J = np.zeros((2, 3))
    for k in range(3):
        xx = x.astype(np.complex128)
        xx[k] += 1j * h
        J[:, k] = np.imag(fun(xx)) / h
    return J


def _sigma_world(scale, quat_wxyz):
    rot = Rotation.from_quat([quat_wxyz[1], quat_wxyz[2], quat_wxyz[3], quat_wxyz[0]]).as_matrix()
    return rot @ np.diag(np.asarray(scale) ** 2) @ rot.T


def _ray_integrals(Sw, M, nrm, d):
    """Full and half (n.X >= 0) integrals of exp(-1/2 X^T Sw^-1 X) along the fibre
    {X : M X = d}, the affine ray through pixel offset d (Eq. 7, Suppl. A.1)."""
    Swi = np.linalg.inv(Sw)
    X0 = M.T @ np.linalg.solve(M @ M.T, d)
    u = np.cross(M[0], M[1])
    u /= np.linalg.norm(u)

    def dens(tau):
        X = X0 + tau * u
        return math.exp(-0.5 * X @ Swi @ X)

    # the integrand is a 1-D Gaussian in tau; integrate over a generous window
    a = u @ Swi @ u
    b = u @ Swi @ X0
    c_tau = -b / a
    s_tau = 1.0 / math.sqrt(a)
    lo, hi = c_tau - 40 * s_tau, c_tau + 40 * s_tau
    full = integrate.quad(dens, lo, hi, epsabs=0, epsrel=1e-13, limit=200)[0]
    nu = nrm @ u
    tstar = -(nrm @ X0) / nu
    tstar = min(max(tstar, lo), hi)
    if nu > 0:      # n.X >= 0 for tau >= tstar
        half = integrate.quad(dens, tstar, hi, epsabs=0, epsrel=1e-13, limit=200)[0]
    else:
        half = integrate.quad(dens, lo, tstar, epsabs=0, epsrel=1e-13, limit=200)[0]
    return full, half


@pytest.mark.parametrize("seed", range(6))
def test_half_integral_matches_quadrature(seed):
    """Eq. 7-8: the oracle's hat G and P equal the ray integrals of the half-Gaussian
    (unfiltered, l = 0), with hat G normalised by the ray integral through the centre."""
    rng = np.random.default_rng(100 + seed)
    vm = _random_view(rng)
    f, W, H = 300.0, 200, 160
    mean = rng.uniform(-0.4, 0.4, 3)
    scale = np.exp(rng.normal(-2.0, 0.6, 3))
    quat = rng.standard_normal(4)
    nrm = rng.standard_normal(3)
    cam = Cam(vm, f, W, H)
    pi = _pixel_map(vm, f, cam.cx, cam.cy)
    M = _jacobian_complex_step(pi, mean)
    Sw = _sigma_world(scale, quat / np.linalg.norm(quat))
    nh = nrm / np.linalg.norm(nrm)
    mu2 = pi(mean)
    sig = np.sqrt(np.diag(M @ Sw @ M.T))
    offs = rng.normal(0, 1.2, size=(12, 2)) * sig
    G, P, mode = oracle.eval_splat(mean, scale, quat, nrm, cam, mu2[0] + offs[:, 0],
                                   mu2[1] + offs[:, 1], lowpass=0.0, fov_clamp=False)
    assert mode == oracle.NORMAL
    full0, _ = _ray_integrals(Sw, M, nh, np.zeros(2))
    for j, d in enumerate(offs):
        full, half = _ray_integrals(Sw, M, nh, d)
        assert G[j] == pytest.approx(full / full0, rel=1e-9, abs=1e-14)
        assert P[j] == pytest.approx(half / full, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_lowpass_is_screen_filter_of_half_footprint(seed):
    """With the 3D-GS low-pass l, P_l * hat G_l / Z_l equals the convolution of the
    unfiltered P_0 * hat G_0 / Z_0 with N(0, l I)  (Z = 2 pi sqrt(det hat Sigma))."""
    rng = np.random.default_rng(200 + seed)
    vm = _random_view(rng)
    f, W, H = 300.0, 200, 160
    lp = float(np.float32(0.3))
    mean = rng.uniform(-0.3, 0.3, 3)
    scale = np.exp(rng.normal(-3.3, 0.4, 3))     # ~1-3 px: the filter matters
    quat = rng.standard_normal(4)
    nrm = rng.standard_normal(3)
    cam = Cam(vm, f, W, H)
    pi = _pixel_map(vm, f, cam.cx, cam.cy)
    M = _jacobian_complex_step(pi, mean)
    Sw = _sigma_world(scale, quat / np.linalg.norm(quat))
    S0 = M @ Sw @ M.T
    Z0 = 2 * math.pi * math.sqrt(np.linalg.det(S0))
    Zl = 2 * math.pi * math.sqrt(np.linalg.det(S0 + lp * np.eye(2)))
    mu2 = pi(mean)
    xs, ws = special.roots_hermite(80)
    E1, E2 = np.meshgrid(xs * math.sqrt(2 * lp), xs * math.sqrt(2 * lp), indexing="ij")
    WW = np.outer(ws, ws) / math.pi
    for d in rng.normal(0, 1.5, size=(4, 2)):
        px = mu2[0] + d[0] - E1.ravel()
        py = mu2[1] + d[1] - E2.ravel()
        G0, P0, _ = oracle.eval_splat(mean, scale, quat, nrm, cam, px, py, lowpass=0.0,
                                      fov_clamp=False)
        conv = float(np.sum(WW.ravel() * G0 * P0)) / Z0
        Gl, Pl, _ = oracle.eval_splat(mean, scale, quat, nrm, cam, [mu2[0] + d[0]],
                                      [mu2[1] + d[1]], lowpass=lp, fov_clamp=False)
        assert Gl[0] * Pl[0] / Zl == pytest.approx(conv, rel=1e-7, abs=1e-12)


def _single_splat_image(sigma, z, f, W, nrm, a1, a2, rgb):
    mean = [0.0, 0.0, z]
    dc = (np.asarray(rgb) - 0.5) * 2.0 * math.sqrt(math.pi)   # Y_00 = 1/(2 sqrt(pi))
    sc = Sc([mean], [[sigma] * 3], [[1, 0, 0, 0]], [nrm], [a1], [a2], dc.reshape(1, 1, 3), 0)
    vm = np.zeros((3, 4)); vm[:, :3] = np.eye(3)
    cam = Cam(vm, f, W, W)
    return oracle.render(sc, cam, lowpass=0.0)


def _closed_form(sigma, z, f, W, nrm, a1, a2, rgb):
    nrm = np.asarray(nrm, np.float64)
    nrm = nrm / np.linalg.norm(nrm)
    ii, jj = np.meshgrid(np.arange(W) + 0.5, np.arange(W) + 0.5, indexing="xy")
    dx, dy = ii - W / 2, jj - W / 2
    G = np.exp(-(dx ** 2 + dy ** 2) * z * z / (2 * f * f * sigma * sigma))
    s = (z / f) * (nrm[0] * dx + nrm[1] * dy)
    if abs(nrm[2]) > 0:
        P = special.ndtr(s / (sigma * abs(nrm[2])))
    else:
        P = np.where(s > 0, 1.0, np.where(s < 0, 0.0, 0.5))
    a = np.minimum(0.99, (a2 + (a1 - a2) * P) * G)
    a = np.where(a < 1 / 255, 0.0, a)
    return np.asarray(rgb)[:, None, None] * a[None], 1.0 - a


@pytest.mark.parametrize("nrm", [[0.3, -0.5, 0.8], [0, 0, 1], [0.6, 0.8, 0.0], [1, 2, -3]])
def test_closed_form_single_splat(nrm):
    """On-axis isotropic splat, identity camera, l = 0: hat Sigma = (f s/z)^2 I,
    w = (z/f)(n1,n2), v = s^2 n3^2, so P = Phi((z/f)(n1 dx + n2 dy)/(s |n3|)).
    n along the view axis gives the mean opacity; n across it gives a hard split."""
    sigma, z, f, W = 0.05, 4.0, 400.0, 48
    a1, a2, rgb = 0.8, 0.15, [0.9, 0.4, 0.2]
    out = _single_splat_image(sigma, z, f, W, nrm, a1, a2, rgb)
    img, T = _closed_form(sigma, z, f, W, nrm, a1, a2, rgb)
    # pixels where a decision sits within 1e-9 of a threshold are not comparable
    ok = out["margin"] > 1e-9
    assert ok.mean() > 0.99
    np.testing.assert_allclose(out["image"][:, ok], img[:, ok], rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["T"][ok], T[ok], rtol=0, atol=1e-12)


def test_normal_along_view_axis_gives_mean_opacity():
    out = _single_splat_image(0.05, 4.0, 400.0, 32, [0, 0, 1], 0.7, 0.1, [1, 1, 1])
    ref = _single_splat_image(0.05, 4.0, 400.0, 32, [0, 0, 1], 0.4, 0.4, [1, 1, 1])
    np.testing.assert_allclose(out["image"], ref["image"], atol=1e-15)


def _config1_variant(equal=False, flip=False):
    sc, cams = scenes.config1()
    s = Sc(sc.means, sc.scales, sc.quats, sc.normals, sc.opac1, sc.opac2, sc.sh, sc.sh_degree)
    if equal:
        s.opac2 = s.opac1.copy()
    if flip:
        s.normals = -s.normals
        s.opac1, s.opac2 = s.opac2.copy(), s.opac1.copy()
    return s, cams[0]


def test_equal_opacities_reduce_to_3dgs_exactly():
    """Sec. 3.2: alpha1 = alpha2 is the 3D-GS kernel.  The HGS image must equal the
    plain-3D-GS image bit for bit in FP64, the normal gradient must vanish exactly
    and the two opacity gradients must sum to the plain opacity gradient."""
    s, cam = _config1_variant(equal=True)
    hgs = oracle.render(s, cam)
    gs = oracle.render(s, cam, plain=True)
    assert np.array_equal(hgs["image"], gs["image"])
    assert np.array_equal(hgs["n_contrib"], gs["n_contrib"])
    g = np.random.default_rng(3).standard_normal(hgs["image"].shape)
    gh = oracle.render_bwd(s, cam, g, proj=hgs["proj"], bins=hgs["bins"])
    gp = oracle.render_bwd(s, cam, g, plain=True, proj=gs["proj"], bins=gs["bins"])
    assert np.all(gh["normals"] == 0.0)
    np.testing.assert_allclose(gh["opac1"] + gh["opac2"], gp["opac1"], rtol=1e-12, atol=1e-13)
    for k in ("means", "scales", "quats", "sh"):
        np.testing.assert_allclose(gh[k], gp[k], rtol=1e-12, atol=1e-13)


def test_complement_symmetry():
    """Sec. 3.2: the complementary half is the same kernel with -n, so
    (n, alpha1, alpha2) and (-n, alpha2, alpha1) render the same image."""
    a, cam = _config1_variant()
    b, _ = _config1_variant(flip=True)
    ra = oracle.render(a, cam)
    rb = oracle.render(b, cam)
    ok = (ra["margin"] > 1e-9) & (rb["margin"] > 1e-9)
    np.testing.assert_allclose(ra["image"][:, ok], rb["image"][:, ok], atol=1e-12, rtol=0)


def test_sh_basis_matches_scipy():
    """Real SH basis: sqrt2 Im Y_l^|m| (m<0), Y_l^0, sqrt2 Re Y_l^m (m>0), with the
    Condon-Shortley phase of scipy's complex harmonics; index l*l + l + m."""
    rng = np.random.default_rng(9)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_eval(3, d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            c = special.sph_harm_y(l, abs(m), theta, phi)
            ref = c.real if m == 0 else (math.sqrt(2) * (c.imag if m < 0 else c.real))
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-13)
    # degree truncation
    Y1 = oracle.sh_eval(1, d)
    assert np.all(Y1[:, 4:] == 0) and np.allclose(Y1[:, :4], Y[:, :4], atol=0)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_binning_against_brute_force(tile):
    """Tiles touched = tiles whose pixel span meets the 3-sigma square [mu - r, mu + r]
    (FP32 endpoints); keys sorted by (tile, depth bits, id); ranges by linear scan."""
    sc, cams = scenes.config1()
    cam = scenes.identity_camera(72, 56, 64.0, 36.0, 28.0)   # ragged tiles at both edges
    pr = oracle.project(sc, cam, tile=tile)
    tx, ty = oracle.grid(cam, tile)
    pairs = []
    for i in range(sc.n):
        if pr["mode"][i] == oracle.CULLED and pr["tiles"][i] == 0:
            continue
        if pr["tiles"][i] == 0:
            continue
        mx, my = pr["canon_mu"][i]
        r = pr["radius"][i]
        lox, hix = np.float32(mx) - np.float32(r), np.float32(mx) + np.float32(r)
        loy, hiy = np.float32(my) - np.float32(r), np.float32(my) + np.float32(r)
        db = int(np.float32(pr["depth"][i]).view(np.uint32))
        for yy in range(ty):
            for xx in range(tx):
                if lox < (xx + 1) * tile[0] and hix >= xx * tile[0] and \
                   loy < (yy + 1) * tile[1] and hiy >= yy * tile[1]:
                    pairs.append((yy * tx + xx, db, i))
    pairs.sort()
    bins = oracle.bin_pairs(pr, cam, tile)
    assert bins["n_pairs"] == len(pairs) == int(pr["tiles"].sum())
    keys = np.array([(t << 32) | d for t, d, _ in pairs], dtype=np.uint64)
    ids = np.array([i for _, _, i in pairs], dtype=np.uint32)
    assert np.array_equal(bins["keys"], keys)
    assert np.array_equal(bins["ids"], ids)
    rng_ref = np.zeros((tx * ty, 2), np.uint32)
    for j, (t, _, _) in enumerate(pairs):
        if j == 0 or pairs[j - 1][0] != t:
            rng_ref[t, 0] = j
        rng_ref[t, 1] = j + 1
    assert np.array_equal(bins["ranges"], rng_ref)


def test_canonical_fields_agree_with_fp64():
    """The FP32 binning fields are the FP64 quantities to FP32 accuracy, and the radius
    covers 3 sqrt(lambda_max) of the FP64 hat Sigma."""
    sc, cams = scenes.config1()
    pr = oracle.project(sc, cams[0])
    ok = pr["mode"] != oracle.CULLED
    np.testing.assert_allclose(pr["canon_mu"][ok], pr["mu2"][ok], rtol=2e-6, atol=1e-4)
    Q = pr["conic"][ok]
    det = Q[:, 0] * Q[:, 2] - Q[:, 1] ** 2
    S = np.stack([Q[:, 2] / det, -Q[:, 1] / det, Q[:, 0] / det], 1)
    np.testing.assert_allclose(pr["canon_abc"][ok], S, rtol=1e-4, atol=1e-5)
    lam = 0.5 * (S[:, 0] + S[:, 2]) + np.sqrt(np.maximum(0.1, 0.25 * (S[:, 0] - S[:, 2]) ** 2 + S[:, 1] ** 2))
    assert np.all(pr["radius"][ok] >= 3 * np.sqrt(lam) * (1 - 1e-5))
    assert np.all(pr["radius"][ok] <= 3 * np.sqrt(lam) + 1 + 1e-3)


def test_compositing_identity_white_over_black():
    """C = sum_i a_i T_i and T_final = prod (1 - a_i): with white splats over black,
    every channel equals 1 - T_final exactly (up to FP64 rounding), and
    T_final is in [1e-4, 1]."""
    sc, cams = scenes.config1()
    s = Sc(sc.means, sc.scales, sc.quats, sc.normals, sc.opac1, sc.opac2,
           np.full((sc.n, 1, 3), 0.5 * 2 * math.sqrt(math.pi)), 0)
    out = oracle.render(s, cams[0])
    assert np.all(out["proj"]["rgb"] == pytest.approx(1.0, abs=1e-15))
    for ch in range(3):
        np.testing.assert_allclose(out["image"][ch], 1.0 - out["T"], atol=1e-13)
    assert out["T"].min() >= 1e-4 and out["T"].max() <= 1.0
    # a brighter splat set bounds the image by max rgb (1 - T)
    sc2, _ = scenes.config1(seed=11)
    o2 = oracle.render(sc2, cams[0])
    mx = o2["proj"]["rgb"][o2["proj"]["mode"] != 0].max(axis=0)
    for ch in range(3):
        assert np.all(o2["image"][ch] <= mx[ch] * (1 - o2["T"]) + 1e-12)


def test_paper_parameter_counts():
    """Sec. 1: 59 parameters per 3D-GS kernel; Sec. 3.2: +3 normal +1 opacity."""
    facts = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))
    sc, _ = scenes.config2(n=10)
    per_kernel = sum(a.reshape(sc.n, -1).shape[1] for a in sc.arrays())
    assert per_kernel == facts["params_per_3dgs_kernel"]["value"] + facts["extra_learned_params_hgs"]["value"]
    assert sc.sh.shape[1] == (facts["sh_degree"]["value"] + 1) ** 2


def test_stacked_splats_stop_rule_and_depth_order():
    """Front-to-back over the depth order with the 3D-GS stop: a splat whose
    compositing would take T below 1e-4 is not composited and ends the list, even
    when a fainter splat behind it would still fit.  Splats are given out of
    depth order; colours identify the order used."""
    f, W = 200.0, 16
    depths = [5.0, 2.0, 4.0, 6.0, 3.0]            # input order (shuffled)
    alphas = [0.95, 0.95, 0.95, 0.10, 0.95]       # by input index
    cols = [[0.1, 0.2, 0.3], [0.9, 0.1, 0.1], [0.2, 0.8, 0.4], [0.5, 0.5, 0.9], [0.3, 0.3, 0.3]]
    sigma = 0.5                                    # ~20 px: G ~ 1 near the centre
    dc = (np.asarray(cols) - 0.5) * 2.0 * math.sqrt(math.pi)
    means = [[0.0, 0.0, z] for z in depths]
    sc = Sc(means, [[sigma] * 3] * 5, [[1, 0, 0, 0]] * 5, [[0, 0, 1]] * 5, alphas, alphas,
            dc.reshape(5, 1, 3), 0)
    vm = np.zeros((3, 4)); vm[:, :3] = np.eye(3)
    out = oracle.render(sc, Cam(vm, f, W, W), lowpass=0.0, composited=True)
    px = py = W // 2                                # centre (8.5, 8.5): d = (0.5, 0.5)
    order = np.argsort(depths)
    T, C, last, comp = 1.0, np.zeros(3), 0, []
    for pos, i in enumerate(order):
        z = depths[i]
        G = math.exp(-(0.5 ** 2 + 0.5 ** 2) * z * z / (2 * f * f * sigma * sigma))
        a = min(0.99, alphas[i] * G)
        if a < 1 / 255:
            continue
        if T * (1 - a) < 1e-4:
            break
        C += np.asarray(cols[i]) * a * T
        T *= 1 - a
        last = pos + 1
        comp.append(pos)
    assert last == 3            # the 4th (depth 5, opaque) stops the list; depth 6 is never reached
    assert np.flatnonzero(out["comp"][:, py, px]).tolist() == comp == [0, 1, 2]
    np.testing.assert_allclose(out["image"][:, py, px], C, atol=1e-13)
    assert out["T"][py, px] == pytest.approx(T, rel=1e-13)
    assert out["n_contrib"][py, px] == last


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_composited_pairs_agree_with_counts(tile):
    """The per-(pair, pixel) composited flags: in every pixel, as many entries of its
    tile's list as the splats composited there, the last one at n_contrib - 1, and
    none in a pixel outside the image (ragged last tiles)."""
    rng = np.random.default_rng(41)
    sc = scenes.scene_uniform(rng, 700, [-1.5, -1.0, 2.5], [1.5, 1.0, 6.0], -3.0, 0.6, 1.5, 1)
    cam = scenes.identity_camera(90, 70, 60.0, 45.0, 35.0)
    out = oracle.render(sc, cam, tile=tile, composited=True, margins=False)
    comp, rng_t = out["comp"], out["bins"]["ranges"].reshape(-1, 2)
    tw, th = tile
    tiles_x = (cam.width + tw - 1) // tw
    assert comp.any()
    for t, (beg, end) in enumerate(rng_t):
        tx, ty = t % tiles_x, t // tiles_x
        for ly in range(th):
            for lx in range(tw):
                px, py = tx * tw + lx, ty * th + ly
                col = comp[beg:end, ly, lx]
                if px >= cam.width or py >= cam.height:
                    assert not col.any()
                    continue
                pos = np.flatnonzero(col)
                assert pos.size == out["n_comp"][py, px]
                assert (pos[-1] + 1 if pos.size else 0) == out["n_contrib"][py, px]
