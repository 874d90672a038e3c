"""Runs a few un-graphed forward+backward steps of the rasterizer on the
scene-scale synthetic workload, for profilers (ncu) and quick timing.

    python -m paper_2406_02720_b300.profile_step [--n 3000000] [--steps 2] [--views 1]
        [--tile 16x16] [--batch 0] [--per-tile]

Each step issues, in order: hgs_project, hgs_bin, hgs_render_fwd,
hgs_rasterize_bwd, hgs_project_bwd (one launch sequence per step, no CUDA graph,
so a profiler sees every kernel launch).  Compositing runs as persistent blocks
over the heaviest-first tile queue, the launch configuration bench.py times
(--per-tile: one block per tile instead).  Prints per-step wall times.
"""
from __future__ import annotations

import argparse
import time


def main(argv=None):
    import torch

    from . import hgs as H
    from . import scenes
    from .rasterizer import Gaussians, Rasterizer

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=3_000_000)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--views", type=int, default=1)
    ap.add_argument("--tile", default="16x16")
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--per-tile", action="store_true")
    args = ap.parse_args(argv)
    tw, th = (int(x) for x in args.tile.split("x"))
    if args.views == 1:
        sc, cams = scenes.config3(n=args.n)
    else:
        sc, cams = scenes.config4(n=args.n, n_views=args.views)
    dL = torch.from_numpy(
        __import__("numpy").concatenate([d.reshape(-1) for d in scenes.upstream_grad(103, cams)])).cuda()
    cfg = H.make_config(tile=(tw, th), batch=args.batch, persistent=not args.per_tile)
    g = Gaussians.from_scene(sc)
    r = Rasterizer(cams, sc.n, cfg)
    r.forward(g)                     # sizes the pair buffers
    grads = Gaussians.empty_like(g)
    torch.cuda.synchronize()
    for k in range(args.steps):
        t0 = time.perf_counter()
        r.clear_status()
        r.forward_async(g)
        r.backward_async(g, dL, grads)
        st = r.read_status()
        t1 = time.perf_counter()
        if st:
            raise SystemExit(f"device status {st}")
        print(f"step {k}: {1e3 * (t1 - t0):.3f} ms wall, {int(r.num_pairs.item())} pairs", flush=True)


if __name__ == "__main__":
    main()
