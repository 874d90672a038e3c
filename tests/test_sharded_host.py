"""Host-side logic of the view-sharded multi-view step, on CPU: the view partition
and the single all-reduce of the flat gradient buffer over two gloo ranks."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2406_02720_b300 import sharded  # noqa: E402
from paper_2406_02720_b300.rasterizer import Gaussians  # noqa: E402


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8, 70])
def test_views_split_once_contiguously_and_evenly(world):
    rng = np.random.default_rng(world)
    pixels = [int(w * h) for w, h in (((640, 360), (1280, 720), (1600, 900), (1920, 1080))[i]
                                      for i in rng.integers(0, 4, 64))]
    shares = [sharded.shard_views(pixels, world, r) for r in range(world)]
    covered = [v for a, b in shares for v in range(a, b)]
    assert covered == list(range(len(pixels)))              # every view once, in order
    per_rank = [sum(pixels[a:b]) for a, b in shares]
    assert max(per_rank) <= sum(pixels) / world + max(pixels)
    with pytest.raises(ValueError):
        sharded.shard_views(pixels, world, world)


def _scene_like(n, sh_degree, value):
    t = {k: torch.full(s, float(value)) for k, s in
         (("means", (n, 3)), ("scales", (n, 3)), ("quats", (n, 4)), ("normals", (n, 3)),
          ("opac1", (n,)), ("opac2", (n,)), ("sh", (n, (sh_degree + 1) ** 2, 3)))}
    return Gaussians(sh_degree=sh_degree, **t)


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2406_02720_b300 import sharded as S
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    g = _scene_like(5, 2, 0.0)
    flat, grads = S.flat_gaussians_like(g)
    # this rank's gradients: distinct values per field and per rank
    for j, k in enumerate(("means", "scales", "quats", "normals", "opac1", "opac2", "sh")):
        getattr(grads, k).fill_(10.0 * j + rank + 1)
    S.all_reduce_grads(flat)
    out[rank] = {k: getattr(grads, k).clone().numpy() for k in ("means", "sh", "opac2")}
    dist.barrier()
    dist.destroy_process_group()


def test_gradients_summed_over_two_gloo_ranks():
    ws = 2
    port = 29500 + os.getpid() % 400
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        assert np.all(res[r]["means"] == 0 * 20.0 + 3.0)           # (10*0 + 1) + (10*0 + 2)
        assert np.all(res[r]["opac2"] == 2 * 50.0 + 3.0)
        assert np.all(res[r]["sh"] == 2 * 60.0 + 3.0)
        assert res[r]["sh"].shape == (5, 9, 3)


def test_flat_buffer_views_cover_it_once():
    g = _scene_like(7, 3, 1.0)
    flat, grads = sharded.flat_gaussians_like(g)
    assert flat.numel() == sum(t.numel() for t in g.tensors())
    for k, t in zip(("means", "scales", "quats", "normals", "opac1", "opac2", "sh"), grads.tensors()):
        assert t.shape == getattr(g, k).shape
        t.fill_(1.0)
    assert torch.all(flat == 1.0)
