"""Mip-Splatting's 3D smoothing filter (paper_2406_02720_b300.mip) against its
definition computed another way: the filtered covariance R S^2 R^T + sigma^2 I and its
determinant ratio from numpy's general matrix routines, and the sampling rate from a
per-camera, per-kernel loop."""
import numpy as np
import torch

from paper_2406_02720_b300 import mip, scenes


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_filtered_scales_and_opacity_factor_match_the_convolved_covariance():
    rng = np.random.default_rng(3)
    n = 200
    scales = np.exp(rng.normal(-3, 1.0, (n, 3)))
    quats = rng.standard_normal((n, 4))
    sig = np.exp(rng.normal(-3.5, 0.8, n))
    o1, o2 = rng.uniform(0.05, 0.95, n), rng.uniform(0.05, 0.95, n)
    eff, e1, e2 = mip.apply_3d_filter(torch.from_numpy(scales), torch.from_numpy(o1), torch.from_numpy(o2),
                                      torch.from_numpy(sig))
    eff, e1, e2 = eff.numpy(), e1.numpy(), e2.numpy()
    for i in range(n):
        R = _rot(quats[i])
        cov = R @ np.diag(scales[i] ** 2) @ R.T
        want = cov + sig[i] ** 2 * np.eye(3)
        got = R @ np.diag(eff[i] ** 2) @ R.T
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)
        f = np.sqrt(np.linalg.det(cov) / np.linalg.det(want))
        np.testing.assert_allclose([e1[i], e2[i]], [o1[i] * f, o2[i] * f], rtol=1e-9)


def test_opacity_factor_gradient_matches_differences():
    rng = np.random.default_rng(4)
    s = torch.tensor(np.exp(rng.normal(-3, 0.5, (5, 3))), requires_grad=True)
    o = torch.tensor(rng.uniform(0.1, 0.9, 5), requires_grad=True)
    sig = torch.tensor(np.exp(rng.normal(-3, 0.5, 5)))
    assert torch.autograd.gradcheck(lambda a, b: mip.apply_3d_filter(a, b, b, sig), (s, o))


def test_sampling_rate_against_a_loop():
    rng = np.random.default_rng(5)
    means = rng.uniform([-3, -2, -1], [3, 2, 9], (400, 3))
    cams = [scenes.identity_camera(320, 200, 250.0)]
    vm = np.zeros((3, 4), np.float32)
    vm[0, 0] = vm[1, 1] = vm[2, 2] = 1.0
    vm[2, 3] = 3.0                                  # a second camera 3 units behind the first
    cams.append(scenes.Camera(vm, 400.0, 400.0, 160.0, 100.0, 320, 200))
    got = mip.max_sampling_rate(torch.from_numpy(means), cams).numpy()
    want = np.zeros(len(means))
    for i, m in enumerate(means):
        for c in cams:
            V = np.asarray(c.viewmat, np.float64)
            t = V[:, :3] @ m + V[:, 3]
            if t[2] > 0.2 and abs(t[0] / t[2]) <= 1.15 * 0.5 * c.width / c.fx and \
                    abs(t[1] / t[2]) <= 1.15 * 0.5 * c.height / c.fy:
                want[i] = max(want[i], max(c.fx, c.fy) / t[2])
    unseen = want == 0
    assert unseen.any() and (~unseen).any()
    want[unseen] = want[~unseen].min()
    np.testing.assert_allclose(got, want, rtol=1e-12)
    sig = mip.filter_sigma(torch.from_numpy(means), cams).numpy()
    np.testing.assert_allclose(sig, np.sqrt(0.2) / want, rtol=1e-12)
