"""The compositing kernels' work counters (hgs_render_stats), which the roofline divides by.

Three of them have a definition outside the kernels and are checked exactly against the
FP64 oracle's per-(pair, pixel) composited flags (Sec. 3.3 blending with the Eq. 10 weight,
1/255 floor, 1e-4 stop):

* composited pairs, forward and backward: the number of set flags;
* backward (warp, splat) visits with more than 12 contributing lanes: for every list entry
  and every 8x4 pixel block of its tile, the block's pixels where the entry is composited
  form the warp's contributing lanes (lane = 8 * row + column in the block);
* backward gradient atomics: per such visit, as many lanes as hold a partial sum after the
  in-warp folds (all contributing lanes up to 12; above 12, the lanes l < 16 with l or
  l + 16 contributing; above 16, the lanes l < 8 with any of l, l + 8, l + 16, l + 24).

The scene is chosen so that FP32 decides every composited flag as FP64 does (no pixel
within the FP32 band of the floor or the stop), so the counts must be equal, not close.
The other counters depend on the kernels' culling and are held to their ordering."""
import numpy as np
import pytest

import oracle
from hgs_testutil import exempt, gpu_render
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def _expected(ref, tile):
    """(composited pairs, folded visits, lane atomics) of one view from its oracle flags."""
    tw, th = tile
    comp = ref["comp"]                                          # [pairs, th, tw] bool
    P = comp.shape[0]
    lanes = comp.reshape(P, th // 4, 4, tw // 8, 8).transpose(0, 1, 3, 2, 4).reshape(P, -1, 32)
    pop = lanes.sum(axis=2)
    by16 = (lanes[..., :16] | lanes[..., 16:]).sum(axis=2)
    by8 = (lanes[..., 0:8] | lanes[..., 8:16] | lanes[..., 16:24] | lanes[..., 24:32]).sum(axis=2)
    atomics = np.where(pop <= 12, pop, np.where(pop <= 16, by16, by8))
    return int(comp.sum()), int((pop > 12).sum()), int(atomics.sum())


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_counters_against_the_oracle(cuda_ok, tile):
    import torch
    rng = np.random.default_rng(47)
    sc = scenes.scene_uniform(rng, 800, [-1.6, -1.1, 2.5], [1.6, 1.1, 6.5], -3.2, 0.6, 1.5, 2)
    cams = [scenes.identity_camera(150, 93, 85.0, 75.0, 46.5, bg=(0.1, 0.2, 0.3)),
            scenes.identity_camera(72, 40, 40.0, 36.0, 20.0)]
    comp = folded = atomics = 0
    for cam in cams:
        ref = oracle.render(sc, cam, tile=tile, composited=True)
        assert not exempt(ref).any()          # every flag decided alike in FP32 and FP64
        c, f, a = _expected(ref, tile)
        comp, folded, atomics = comp + c, folded + f, atomics + a
    out = gpu_render(sc, cams, tile=tile)
    r = out["rast"]
    st = r.stats(torch.ones_like(r.image))
    assert st["fwd_comp"] == comp and st["bwd_contrib"] == comp, (st, comp)
    assert st["bwd_warp_red"] == folded, (st["bwd_warp_red"], folded)
    assert st["bwd_atomic"] == atomics, (st["bwd_atomic"], atomics)
    assert st["fwd_comp"] <= st["fwd_full"] <= st["fwd_visit"]
    assert st["bwd_contrib"] <= st["bwd_full"] <= st["bwd_visit"]
    assert comp > 10000 and folded > 100 and atomics < comp
