"""The oracle's hand-written FP64 adjoint against central finite differences of
its own FP64 forward (CPU only).

Loss L = sum(g * image) for a fixed random g.  Coordinates whose step-h and
step-h/2 difference quotients disagree sit on a threshold or a binning edge
(1/255 floor, 1e-4 stop, tile rect) where the derivative does not exist; they
are skipped and counted.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_02720_b300 import scenes


class Sc:
    def __init__(self, d, deg):
        self.__dict__.update(d)
        self.sh_degree = deg

    def copy(self):
        return Sc({k: np.array(v, np.float64, copy=True) for k, v in self.__dict__.items()
                   if k != "sh_degree"}, self.sh_degree)


def _scene(seed, n=12, deg=3, W=40, H=32):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.9, 0.9, n), rng.uniform(-0.7, 0.7, n), rng.uniform(2.5, 5, n)], 1)
    scales = np.exp(rng.normal(-2.6, 0.4, (n, 3)))
    quats = rng.standard_normal((n, 4))
    normals = rng.standard_normal((n, 3))
    o1 = 1 / (1 + np.exp(-rng.normal(0, 1, n)))
    o2 = 1 / (1 + np.exp(-rng.normal(0, 1, n)))
    sh = rng.normal(0, 0.3, (n, (deg + 1) ** 2, 3))
    sh[:, 0, :] += 0.6
    # two big splats beyond the +-1.3 tan(fov/2) clamp that still reach the image
    means[0] = [2.6, 0.1, 3.0]
    scales[0] = [1.2, 1.0, 0.9]
    means[1] = [-0.2, -2.4, 3.0]
    scales[1] = [0.9, 1.1, 1.0]
    sc = Sc(dict(means=means, scales=scales, quats=quats, normals=normals, opac1=o1, opac2=o2,
                 sh=sh), deg)
    vm = np.zeros((3, 4))
    ang = 0.2
    vm[:, :3] = [[math.cos(ang), 0, math.sin(ang)], [0, 1, 0], [-math.sin(ang), 0, math.cos(ang)]]
    vm[:, 3] = [0.05, 0.02, 0.3]
    cam = scenes.Camera(vm, 40.0, 42.0, 19.0, 17.0, W, H, bg=(0.2, 0.1, 0.3))
    g = rng.standard_normal((3, H, W))
    return sc, cam, g


def _loss(sc, cam, g, **kw):
    return float(np.sum(oracle.render(sc, cam, **kw)["image"] * g))


@pytest.mark.parametrize("seed,plain,mip", [(0, False, False), (1, False, False), (2, True, False),
                                             (3, False, True)])
def test_adjoint_matches_central_differences(seed, plain, mip):
    """mip: the opacity compensation of the Mip-Splatting 2D filter, with its gradient
    through det hat Sigma_0 / det hat Sigma into the geometry."""
    sc, cam, g = _scene(seed)
    kw = dict(tile=(16, 16), plain=plain, mip=mip)
    out = oracle.render(sc, cam, **kw)
    # both clamp branches of the Jacobian are exercised: splats 0 and 1 have their
    # centre beyond 1.3 tan(fov/2) and still cover tiles
    pr = out["proj"]
    for i, (ax, f, W) in ((0, (0, cam.fx, cam.width)), (1, (1, cam.fy, cam.height))):
        t = cam.viewmat[:, :3] @ sc.means[i] + cam.viewmat[:, 3]
        assert abs(t[ax] / t[2]) > 1.3 * 0.5 * W / f
        assert pr["mode"][i] != 0 and pr["tiles"][i] > 0
    ad = oracle.render_bwd(sc, cam, g, proj=out["proj"], bins=out["bins"], **kw)
    # rounding noise of a difference quotient: a few ulps of sum|g*image| over 2h
    lsum = float(np.sum(np.abs(out["image"] * g)))
    checked = skipped = 0
    for name in ("means", "scales", "quats", "normals", "opac1", "opac2", "sh"):
        A = getattr(sc, name)
        gref = ad[name].reshape(A.shape)
        floor = 1e-4 * max(np.abs(gref).max(), 1e-8)
        flat_idx = np.ndindex(*A.shape)
        for idx in flat_idx:
            if name == "sh" and idx[1] > 4 and (idx[0] % 3):   # thin out SH coordinates
                continue
            if plain and name in ("normals", "opac2"):
                continue
            x0 = A[idx]
            est = []
            for h in (1e-6 * max(1.0, abs(x0)), 0.5e-6 * max(1.0, abs(x0))):
                A[idx] = x0 + h
                lp = _loss(sc, cam, g, **kw)
                A[idx] = x0 - h
                lm = _loss(sc, cam, g, **kw)
                A[idx] = x0
                est.append((lp - lm) / (2 * h))
            scale = max(abs(est[0]), abs(gref[idx]), floor)
            noise = 8 * 2.2e-16 * lsum / (1e-6 * max(1.0, abs(x0)))
            if abs(est[0] - est[1]) > 1e-5 * scale + 3 * noise:
                skipped += 1
                continue
            checked += 1
            assert abs(est[0] - gref[idx]) <= 1e-6 * scale + noise, (name, idx, est, gref[idx])
    assert checked > 300 and skipped <= 0.02 * (checked + skipped), (checked, skipped)


def test_screen_space_gradients_match_differences():
    """The per-splat screen-space gradients (grad2d) against differences of the
    compositing step alone, with the projection held fixed."""
    sc, cam, g = _scene(5, n=10, deg=1)
    out = oracle.render(sc, cam)
    ad = oracle.render_bwd(sc, cam, g, proj=out["proj"], bins=out["bins"])["grad2d"]
    pr = out["proj"]
    fields = [("mu2", 0), ("mu2", 1), ("conic", 0), ("conic", 1), ("conic", 2), ("wp", 0),
              ("wp", 1), ("opac1", None), ("opac2", None), ("rgb", 0), ("rgb", 1), ("rgb", 2)]
    lsum = float(np.sum(np.abs(out["image"] * g)))
    checked = 0
    for i in range(sc.means.shape[0]):
        if pr["mode"][i] != oracle.NORMAL:
            continue
        for j, (key, col) in enumerate(fields):
            arr = pr[key]
            x0 = arr[i] if col is None else arr[i, col]
            h = 1e-6 * max(1.0, abs(x0))
            vals = []
            for s in (+1, -1):
                if col is None:
                    arr[i] = x0 + s * h
                else:
                    arr[i, col] = x0 + s * h
                r = oracle.render(sc, cam, proj=pr, bins=out["bins"])
                vals.append(float(np.sum(r["image"] * g)))
            if col is None:
                arr[i] = x0
            else:
                arr[i, col] = x0
            fd = (vals[0] - vals[1]) / (2 * h)
            scale = max(abs(fd), abs(ad[i, j]), 1e-6)
            noise = 8 * 2.2e-16 * lsum / h
            assert abs(fd - ad[i, j]) <= 2e-6 * scale + noise, (i, key, col, fd, ad[i, j])
            checked += 1
    assert checked > 60
