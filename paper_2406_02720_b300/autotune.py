"""Picks the tile shape and shared-memory batch size of the compositing kernels
by timing a captured forward+backward step for each candidate, and caches the
choice in a JSON file keyed by (GPU name, splat-count bucket, view sizes).

The tile shape changes the rendered image (tiles are culled by the 3-sigma
square, not per pixel), so the choice is the caller's to accept; every
supported shape is parity-tested against the oracle run with that shape.
"""
from __future__ import annotations

import json
import math
import os

# (tile shape, batch): batch 0 takes each compositing kernel's own default (forward 128
# splats, or 64 at 8x8; backward 224, or 64 at 8x8), a non-zero batch is used by both
CANDIDATES = [((16, 16), 0), ((16, 16), 128), ((32, 8), 0), ((32, 8), 128), ((8, 8), 0), ((8, 8), 128)]


def n_bucket(n: int) -> int:
    """Splat counts are bucketed to the nearest power of two."""
    return 1 << max(0, round(math.log2(max(n, 1))))


def cache_key(gpu_name: str, n: int, sizes, persistent: bool) -> str:
    hist = {}
    for w, h in sizes:
        hist[f"{w}x{h}"] = hist.get(f"{w}x{h}", 0) + 1
    views = ",".join(f"{k}:{v}" for k, v in sorted(hist.items()))
    # the candidate set is part of the key: a choice made among other candidates is stale
    cands = ";".join(f"{t[0]}x{t[1]}/{b}" for t, b in CANDIDATES)
    return f"{gpu_name}|n~{n_bucket(n)}|{views}|{'persistent' if persistent else 'per-tile'}|{cands}"


def load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def store(path, key, entry):
    if not path:
        return
    data = load(path)
    data[key] = entry
    tmp = path + ".tmp"
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(timings):
    """The fastest candidate: list of (tile, batch, ms) -> (tile, batch)."""
    best = min(timings, key=lambda t: t[2])
    return tuple(best[0]), int(best[1])


def tune(cams, g, dL_packed, candidates=CANDIDATES, steps=5, cache_path=None, persistent=True, device="cuda"):
    """Times each candidate's captured fwd+bwd step; returns (tile, batch, timings).
    A cached result for the same key is returned without timing."""
    import torch

    from .multiview import BatchedStep, time_replays
    name = torch.cuda.get_device_name(torch.device(device))
    key = cache_key(name, g.n, [(c.width, c.height) for c in cams], persistent)
    cached = load(cache_path).get(key)
    if cached:
        return tuple(cached["tile"]), int(cached["batch"]), cached["timings"]
    timings = []
    for tile, batch in candidates:
        step = BatchedStep(cams, g, dL_packed, tile=tile, batch=batch, device=device)
        if not persistent:
            raise ValueError("tuning is defined for the persistent (view, tile) path")
        ms = time_replays(step, steps)
        if step.status():
            raise RuntimeError(f"device status during tuning of {tile}/{batch}")
        timings.append((list(tile), batch, ms))
        del step
        torch.cuda.empty_cache()
    tile, batch = pick(timings)
    store(cache_path, key, {"tile": list(tile), "batch": batch, "timings": timings})
    return tile, batch, timings
