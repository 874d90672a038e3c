"""End to end through autograd: fitting a perturbed copy of a hidden scene to its renders
with Adam (paper_2406_02720_b300.train) lowers the L1 loss, every parameter receives a
finite gradient, and the autograd gradients equal the direct adjoint call."""
import numpy as np
import pytest

from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def _setup(seed=51):
    rng = np.random.default_rng(seed)
    hidden = scenes.scene_uniform(rng, 1500, [-1.2, -0.9, 2.5], [1.2, 0.9, 6.0], -3.0, 0.5, 1.5, 1)
    cams = [scenes.identity_camera(128, 96, 100.0),
            scenes.look_at_camera([0.8, 0.3, -0.5], [0.0, 0.0, 4.0], [0.0, 1.0, 0.0], 128, 96, 100.0)]
    init = hidden.subset(np.arange(hidden.n))
    init.means += rng.normal(0, 0.03, init.means.shape).astype(np.float32)
    init.opac1[:] = 0.5
    init.opac2[:] = 0.5
    init.normals[:] = rng.standard_normal(init.normals.shape).astype(np.float32)
    return hidden, init, cams


def test_fit_lowers_the_loss(cuda_ok):
    from paper_2406_02720_b300 import train
    hidden, init, cams = _setup()
    target = train.render_targets(hidden, cams)
    model, losses = train.fit(init, cams, target, iters=150)
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.6 * losses[0], (losses[0], losses[-1])
    for p in model.parameters():
        assert p.grad is None or bool(p.grad.isfinite().all())


def test_fit_mip_splatting_hgs_lowers_the_loss(cuda_ok):
    """Mip-Splatting-HGS (3D filter in the activation, 2D filter in the rasterizer)
    fitted to targets rendered the same way."""
    from paper_2406_02720_b300 import hgs as H, train
    hidden, init, cams = _setup(53)
    cfg = H.make_config(mip=True, lowpass=0.1)
    target = train.render_targets(hidden, cams, cfg)
    model, losses = train.fit(init, cams, target, iters=150, mip=True)
    assert model.filter_sigma is not None and bool((model.filter_sigma > 0).all())
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.6 * losses[0], (losses[0], losses[-1])


def test_autograd_matches_the_adjoint_call(cuda_ok):
    import torch
    from paper_2406_02720_b300 import hgs as H
    from paper_2406_02720_b300.rasterizer import Gaussians, HGSRasterize, Rasterizer
    hidden, _, cams = _setup(52)
    g = Gaussians.from_scene(hidden)
    leaves = [t.clone().requires_grad_(True) for t in g.tensors()]
    r = Rasterizer(cams, hidden.n, H.make_config())
    img = HGSRasterize.apply(r, g.sh_degree, *leaves)
    dL = torch.randn_like(img)
    (img * dL).sum().backward()
    r2 = Rasterizer(cams, hidden.n, H.make_config())
    r2.forward(g)
    direct = r2.backward(g, dL)
    for leaf, d in zip(leaves, direct.tensors()):
        assert torch.allclose(leaf.grad, d, rtol=1e-4, atol=1e-6 * float(d.abs().max()) + 1e-12)
