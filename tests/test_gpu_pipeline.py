"""The backward compositing pipeline's bounded wait.

Inside a block of the backward, one warp stages each tile's list and the others
walk it, synchronised by shared-memory mbarriers; every wait gives up after about
a second, sets HGS_DEV_TIMEOUT and returns.  The self-test waits on an mbarrier
that nothing completes (a wait that must run out) and checks the status the host
reads, the time it took, and that the context still renders and differentiates
a scene correctly afterwards."""
import time

import numpy as np
import pytest

import oracle
from hgs_testutil import check_grads, gpu_render, masked_upstream
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_reports(cuda_ok):
    import torch
    from paper_2406_02720_b300 import hgs as H
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H.hgs_selftest_wait(status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert int(status.item()) == H.HGS_DEV_TIMEOUT
    assert 0.5 < waited < 10.0
    with pytest.raises(RuntimeError):
        H.hgs_selftest_wait(None, 0)


def test_backward_after_a_timed_out_wait(cuda_ok):
    """The device stays usable: a full forward and backward afterwards is clean and
    matches the FP64 adjoint."""
    import torch
    from paper_2406_02720_b300 import hgs as H
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    H.hgs_selftest_wait(status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(status.item()) == H.HGS_DEV_TIMEOUT
    rng = np.random.default_rng(31)
    sc = scenes.scene_uniform(rng, 800, [-1.3, -0.8, 2.5], [1.3, 0.8, 6], -3.3, 0.5, 1.5, 3)
    cams = [scenes.identity_camera(160, 96, 90.0, 80.0, 48.0, bg=(0.3, 0.2, 0.1))]
    ref = oracle.render(sc, cams[0])
    dL = masked_upstream(scenes.upstream_grad(102, cams), [ref])
    out = gpu_render(sc, cams, dL=dL)
    assert out["rast"].read_status() == 0
    g = oracle.render_bwd(sc, cams[0], dL[0], proj=ref["proj"], bins=ref["bins"])
    for k in ("means", "scales", "quats", "normals", "opac1", "opac2", "sh"):
        check_grads(out["grads"][k], g[k], ref["touched"], label=k, err=g["err_" + k])
