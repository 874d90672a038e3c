"""Pins of the oracle's Mip-Splatting-HGS mode (mip=True): the screen-space low-pass
as Mip-Splatting's 2D filter, i.e. a normalised convolution rather than a dilation.

By total probability, convolving the undilated half-Gaussian footprint
(alpha2 + (alpha1 - alpha2) P_0(d)) hat G_0(d) with the normalised N(0, l I) gives
exactly sqrt(det hat Sigma_0 / det hat Sigma) (alpha2 + (alpha1 - alpha2) P(d)) hat G(d),
with P and hat G taken from the dilated hat Sigma = hat Sigma_0 + l I.  The test
computes that convolution by 2-D Gauss-Hermite quadrature from the oracle's own l = 0
evaluation, so a wrong factor, a wrong determinant or a P that ignores the low-pass
fails it.  The plain dilation (mip=False) is checked to miss it."""
import numpy as np
import pytest

import oracle
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.filterwarnings("ignore")

CAM = scenes.identity_camera(256, 256, 300.0)
LP = 0.3


class One:
    def __init__(self, m, s, q, n, a1, a2):
        self.means = np.array([m], np.float64)
        self.scales = np.array([s], np.float64)
        self.quats = np.array([q], np.float64)
        self.normals = np.array([n], np.float64)
        self.opac1 = np.array([a1], np.float64)
        self.opac2 = np.array([a2], np.float64)
        self.sh = np.zeros((1, 1, 3))
        self.sh_degree = 0


def _splats(seed, k=6):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        m = [rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(3, 5)]
        s = np.exp(rng.normal(-4.3, 0.5, 3))          # footprints of ~0.5 to 4 px
        q = rng.standard_normal(4)
        n = rng.standard_normal(3)
        out.append(One(m, s, q, n, rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9)))
    return out


def _weight(sp, px, py, lowpass):
    G, P, mode = oracle.eval_splat(sp.means[0], sp.scales[0], sp.quats[0], sp.normals[0], CAM, px, py,
                                   lowpass=lowpass)
    assert mode == oracle.NORMAL
    return (sp.opac2[0] + (sp.opac1[0] - sp.opac2[0]) * P) * G


def _convolved(sp, px, py, nodes=160):
    """(undilated half-Gaussian weight) * N(0, LP I), by Gauss-Hermite quadrature."""
    x, w = np.polynomial.hermite_e.hermegauss(nodes)     # weight exp(-x^2 / 2)
    ex, ey = np.meshgrid(x, x, indexing="ij")
    ww = np.outer(w, w) / (2 * np.pi)
    sd = np.sqrt(float(np.float32(LP)))                    # the low-pass the oracle receives
    out = np.zeros(px.size)
    for j in range(px.size):
        f = _weight(sp, px[j] - sd * ex.ravel(), py[j] - sd * ey.ravel(), 0.0)
        out[j] = np.sum(ww.ravel() * f)
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_mip_weight_is_the_convolved_half_footprint(seed):
    for sp in _splats(seed):
        pr = oracle.project(sp, CAM, tile=(16, 16), lowpass=LP, mip=True)
        plain = oracle.project(sp, CAM, tile=(16, 16), lowpass=LP, mip=False)
        c = pr["comp"][0]
        assert 0.0 < c < 1.0 and plain["comp"][0] == 1.0
        assert pr["opac1"][0] == pytest.approx(c * sp.opac1[0], rel=1e-15)
        mu = pr["mu2"][0]
        rng = np.random.default_rng(seed + 7)
        # pixel offsets within ~2.5 sigma of the dilated footprint
        a, b, cc = np.linalg.inv(np.array([[pr["conic"][0][0], pr["conic"][0][1]],
                                           [pr["conic"][0][1], pr["conic"][0][2]]]))[[0, 0, 1], [0, 1, 1]]
        px = mu[0] + rng.uniform(-2.5, 2.5, 12) * np.sqrt(a)
        py = mu[1] + rng.uniform(-2.5, 2.5, 12) * np.sqrt(cc)
        want = _convolved(sp, px, py)
        got = c * _weight(sp, px, py, LP)
        assert np.abs(got - want).max() <= 1e-11 * want.max(), (got, want)
        # the plain dilation is not the convolution: it misses by the factor 1 / c
        assert np.abs(_weight(sp, px, py, LP) - want).max() > 1e-3 * want.max()


def test_mip_without_lowpass_is_the_plain_kernel():
    sc, cams = scenes.config1()
    a = oracle.render(sc, cams[0], lowpass=0.0, mip=True)
    b = oracle.render(sc, cams[0], lowpass=0.0, mip=False)
    assert np.all(a["proj"]["comp"][a["proj"]["mode"] != oracle.CULLED] == 1.0)
    assert np.array_equal(a["image"], b["image"])


def test_mip_compensation_only_darkens():
    sc, cams = scenes.config1()
    a = oracle.render(sc, cams[0], mip=True)
    b = oracle.render(sc, cams[0], mip=False)
    live = a["proj"]["mode"] != oracle.CULLED
    c = a["proj"]["comp"][live]
    assert np.all(c > 0) and np.all(c < 1)
    # with a black background, every pixel's coverage can only drop (T can only rise)
    assert np.all(a["T"] >= b["T"] - 1e-12)
