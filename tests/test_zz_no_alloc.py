"""hgs_bin_static, the binning entry point that keeps its scratch in a fixed
device array inside the library, for callers that must not allocate device
memory (a plug-in whose host application owns the memory budget, a real-time
loop that cannot afford a driver allocation).  Its outputs must equal those of
hgs_bin, which takes caller scratch, bit for bit (binning is integer work), on
two calls in a row with different inputs, the second running over the scratch
the first left behind; and a call after the first must not change the device's
free memory or PyTorch's allocated bytes.

This file is collected last so that a run stopping at the first failure has run
every other test before it; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2406_02720_b300 import hgs as H
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _scene(seed, n):
    rng = np.random.default_rng(seed)
    sc = scenes.scene_uniform(rng, n, [-1.6, -1.2, 2], [1.6, 1.2, 7], -3.0, 0.6, 1.2, 1)
    return sc, [scenes.identity_camera(100, 75, 70.0, 51.0, 36.5)]


def _static_bin(r, capacity):
    import torch
    keys = torch.full((capacity,), -1, dtype=torch.int64, device="cuda")
    ids = torch.full((capacity,), -1, dtype=torch.int32, device="cuda")
    ranges = torch.full((r.total_tiles, 2), -1, dtype=torch.int32, device="cuda")
    num = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    H.hgs_bin_static(r.proj_struct(), r.n, r.cams_host, r.n_views, r.cfg, capacity, _vp(keys), _vp(ids),
                     _vp(ranges), _vp(num), _vp(status), stream)
    torch.cuda.synchronize()
    free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    k = int(num.item())
    return (keys[:k].cpu().numpy(), ids[:k].cpu().numpy(), ranges.cpu().numpy(), int(status.item()),
            free1 - free0, alloc1 - alloc0)


def test_static_scratch_binning_matches_caller_scratch(cuda_ok):
    from paper_2406_02720_b300.rasterizer import Gaussians, Rasterizer
    for call, (seed, n) in enumerate(((21, 1500), (22, 900))):     # two calls in a row, different sizes
        sc, cams = _scene(seed, n)
        r = Rasterizer(cams, sc.n, H.make_config(), keep_keys=True)
        r.forward(Gaussians.from_scene(sc))          # projection + hgs_bin with caller scratch
        k_ref, i_ref = (x.cpu().numpy() for x in r.sorted_pairs())
        rng_ref = r.ranges.cpu().numpy()
        assert k_ref.size > 500
        need = H.hgs_bin_workspace_size(r.n, r.n_views, r.capacity)
        assert need <= H.HGS_BIN_STATIC_SCRATCH_BYTES
        keys, ids, ranges, status, d_free, d_alloc = _static_bin(r, r.capacity)
        assert status == 0
        assert d_alloc == 0                          # nothing from PyTorch's allocator
        if call > 0:
            # the first call in a process may load the module that holds the array;
            # after that a call takes no device memory at all
            assert d_free == 0, d_free
        assert np.array_equal(keys, k_ref)
        assert np.array_equal(ids, i_ref)
        assert np.array_equal(ranges, rng_ref)


def test_static_scratch_rejects_sizes_beyond_its_limit(cuda_ok):
    sc, cams = _scene(23, 100)
    from paper_2406_02720_b300.rasterizer import Rasterizer
    r = Rasterizer(cams, sc.n, H.make_config())
    too_many = H.HGS_BIN_STATIC_SCRATCH_BYTES // 8       # keys alone would not fit
    assert H.hgs_bin_workspace_size(r.n, r.n_views, too_many) > H.HGS_BIN_STATIC_SCRATCH_BYTES
    st = H.lib().hgs_bin_static(ctypes.byref(r.proj_struct()), r.n, r.cams_host, r.n_views, ctypes.byref(r.cfg),
                                too_many, ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256),
                                ctypes.c_void_p(256), None, None)
    assert st == H.HGS_ERR_CAPACITY
