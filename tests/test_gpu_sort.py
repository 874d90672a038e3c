"""The radix sort over many partitions.

Each pass of the sort ranks 4096-key partitions, each placed by the digit counts
of the partitions before it.  These tests sort scenes large enough for many
partitions in both stages (depth keys and pairs, each with a ragged last
partition; 885 pair partitions in the larger case, more than the 592 downsweep
blocks a B300 holds at once)
and compare the pairs and tile ranges with the oracle's plain lexicographic sort
bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def _scene(n, seed):
    rng = np.random.default_rng(seed)
    sc = scenes.scene_uniform(rng, n, [-2.4, -1.4, 2], [2.4, 1.4, 9], -3.6, 0.5, 1.0, 1)
    return sc, [scenes.identity_camera(640, 360, 500.0, 319.5, 179.5)]


def _gpu_bin(sc, cams, tile, capacity):
    """Projection and binning alone through the C ABI: sorted keys, ids, ranges, status."""
    import torch
    from paper_2406_02720_b300 import hgs as H
    from paper_2406_02720_b300.rasterizer import Gaussians, Rasterizer
    r = Rasterizer(cams, sc.n, H.make_config(tile=tile), pair_capacity=capacity, keep_keys=True)
    g = Gaussians.from_scene(sc)
    r.clear_status()
    r.project(g)
    r.bin()
    torch.cuda.synchronize()
    k, i = r.sorted_pairs()
    return dict(keys=k.cpu().numpy().view(np.uint64), ids=i.cpu().numpy().view(np.uint32),
                ranges=r.ranges.cpu().numpy().view(np.uint32), status=r.read_status())


@pytest.mark.parametrize("n,tile", [(50_001, (16, 16)), (200_003, (8, 8))])
def test_binning_many_partitions_bit_exact(cuda_ok, n, tile):
    sc, cams = _scene(n, 5 + n % 7)
    ref = oracle.bin_pairs(oracle.project(sc, cams[0], tile=tile, errmat=False), cams[0], tile)
    out = _gpu_bin(sc, cams, tile, ref["n_pairs"] + 5000)
    assert out["status"] == 0
    assert n // 4096 >= 12                         # many depth partitions
    assert ref["n_pairs"] // 4096 >= 30 and ref["n_pairs"] % 4096 != 0
    assert out["keys"].size == ref["n_pairs"]
    assert np.array_equal(out["keys"], ref["keys"])
    assert np.array_equal(out["ids"], ref["ids"])
    assert np.array_equal(out["ranges"], ref["ranges"])


@pytest.mark.parametrize("z0,z1,passes", [(4.0, 4.0, 1), (4.0, 4.003, 2), (4.0, 7.0, 3)])
def test_depth_passes_follow_the_key_range(cuda_ok, z0, z1, passes):
    """The depth stage sorts key - min in as many 8-bit passes as the drawn splats'
    key range needs (all four are launched; the rest return at once).  Depths in
    [z0, z1] on the optical-axis camera need `passes` passes; z0 = z1 gives equal keys,
    whose order is the splat index alone.  Pairs and ranges bit-exact."""
    import bench
    rng = np.random.default_rng(91)
    n = 50_001
    sc = scenes.scene_uniform(rng, n, [-2.4, -1.4, z0], [2.4, 1.4, z1], -3.6, 0.5, 1.0, 1)
    if z0 == z1:
        sc.means[:, 2] = np.float32(z0)
    cams = [scenes.identity_camera(640, 360, 500.0, 319.5, 179.5)]
    pr = oracle.project(sc, cams[0], errmat=False)
    assert bench.depth_sort_passes(pr["depth"], pr["tiles"]) == passes
    ref = oracle.bin_pairs(pr, cams[0], (16, 16))
    out = _gpu_bin(sc, cams, (16, 16), ref["n_pairs"] + 5000)
    assert out["status"] == 0
    assert out["keys"].size == ref["n_pairs"] > 4096 * 12
    assert np.array_equal(out["keys"], ref["keys"])
    assert np.array_equal(out["ids"], ref["ids"])
    assert np.array_equal(out["ranges"], ref["ranges"])
