"""The view-sharded multi-view step (paper_2406_02720_b300.sharded) on two ranks: two
processes, both on cuda:0, exchanging gradients over gloo (one all-reduce of the flat
gradient buffer; gloo copies CUDA tensors through the host, and no kernel of one rank
waits on the other).  Each rank renders its share of four uneven views; after the
all-reduce both ranks hold the gradient of the whole step, which must equal the
single-process batched step over all four views (up to the order of FP32 atomics)
and the FP64 oracle's sum over the views."""
import os
import sys
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from hgs_testutil import check_grads, masked_upstream
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = ("means", "scales", "quats", "normals", "opac1", "opac2", "sh")


def _setup():
    rng = np.random.default_rng(52)
    sc = scenes.scene_uniform(rng, 2500, [-2, -2, -2], [2, 2, 2], -3.4, 0.6, 1.5, 3)
    cams = scenes.fibonacci_cameras(4, radius=6.0, resolutions=[(96, 64), (160, 90), (64, 64), (200, 120)])
    return sc, cams


def _rank_main(rank, ws, port, dl_path, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2406_02720_b300.rasterizer import Gaussians
    from paper_2406_02720_b300.sharded import ShardedStep
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sc, cams = _setup()
    z = np.load(dl_path)
    dL = [z[f"dL{v}"] for v in range(len(cams))]
    g = Gaussians.from_scene(sc)
    step = ShardedStep(cams, g, dL)
    for _ in range(2):                      # twice: every step starts from zero gradients
        step.replay()
    torch.cuda.synchronize()
    assert step.status() == 0
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), start=step.start, stop=step.stop,
             **{k: getattr(step.grads, k).cpu().numpy() for k in FIELDS})
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_view_sharded_step(cuda_ok):
    import torch
    from paper_2406_02720_b300.multiview import BatchedStep, packed_upstream
    from paper_2406_02720_b300.rasterizer import Gaussians
    sc, cams = _setup()
    refs = [oracle.render(sc, c) for c in cams]
    dL = masked_upstream(scenes.upstream_grad(9, cams), refs)
    with tempfile.TemporaryDirectory() as tmp:
        dl_path = os.path.join(tmp, "dl.npz")
        np.savez(dl_path, **{f"dL{v}": d for v, d in enumerate(dL)})
        port = 29900 + os.getpid() % 90
        mp.spawn(_rank_main, args=(2, port, dl_path, tmp), nprocs=2, join=True)
        ranks = [dict(np.load(os.path.join(tmp, f"rank{r}.npz"))) for r in range(2)]
    # the two ranks rendered disjoint, covering shares and hold the same reduced gradient
    assert (int(ranks[0]["start"]), int(ranks[0]["stop"])) == (0, int(ranks[1]["start"]))
    assert int(ranks[1]["stop"]) == len(cams) and 0 < int(ranks[0]["stop"]) < len(cams)
    for k in FIELDS:
        assert np.array_equal(ranks[0][k], ranks[1][k])
    # single-process batched step over all views
    g = Gaussians.from_scene(sc)
    b = BatchedStep(cams, g, packed_upstream(dL, "cuda"))
    b.replay()
    torch.cuda.synchronize()
    tot = None
    for c, d, ref in zip(cams, dL, refs):
        gr = oracle.render_bwd(sc, c, d, proj=ref["proj"], bins=ref["bins"])
        tot = gr if tot is None else {k: tot[k] + gr[k] for k in tot}
    touched = np.logical_or.reduce([r["touched"] for r in refs])
    for k in FIELDS:
        got = ranks[0][k].astype(np.float64)
        gb = getattr(b.grads, k).cpu().numpy().astype(np.float64)
        # float atomics and the all-reduce sum in different orders
        np.testing.assert_allclose(got, gb, rtol=1e-3, atol=1e-5 * np.abs(gb).max())
        check_grads(got, tot[k], touched, label=f"sharded {k}", err=tot["err_" + k])
