"""The C-ABI library loads without a GPU, exports every function include/hgs.h
declares, and rejects bad arguments on the host (no kernel is launched)."""
import ctypes

import numpy as np

from paper_2406_02720_b300 import hgs as H
from paper_2406_02720_b300 import scenes


def test_library_exports_every_declared_symbol():
    L = H.lib()
    names = H.declared_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(L, name), name
    for required in ("hgs_project", "hgs_bin", "hgs_render_fwd", "hgs_render_bwd"):
        assert required in names
    assert H.hgs_version() == 2
    assert H.hgs_status_string(H.HGS_ERR_INVALID) == "invalid argument"


def test_layout_and_workspace_sizes():
    cams = [scenes.identity_camera(100, 75, 64.0), scenes.identity_camera(1920, 1080, 1500.0)]
    for tile, want in (((16, 16), 7 * 5 + 120 * 68), ((8, 8), 13 * 10 + 240 * 135), ((32, 8), 4 * 10 + 60 * 135)):
        cfg = H.make_config(tile=tile)
        tiles, pix = H.hgs_layout(H.make_cameras(cams), 2, cfg)
        assert tiles == want
        assert pix == 100 * 75 + 1920 * 1080
    assert H.hgs_bin_workspace_size(1000, 1, 10000) > 10000 * 12
    assert H.hgs_bin_workspace_size(1000, 1, 20000) > H.hgs_bin_workspace_size(1000, 1, 10000)


def test_host_validation_rejects_bad_arguments():
    L = H.lib()
    cams = H.make_cameras([scenes.identity_camera(64, 64, 64.0)])
    bad_tile = H.make_config(tile=(12, 12))
    assert L.hgs_layout(cams, 1, ctypes.byref(bad_tile), None, None) == H.HGS_ERR_INVALID
    bad_batch = H.make_config(batch=48)
    assert L.hgs_layout(cams, 1, ctypes.byref(bad_batch), None, None) == H.HGS_ERR_INVALID
    bad_rect = H.make_config(rect_mode=3)
    assert L.hgs_layout(cams, 1, ctypes.byref(bad_rect), None, None) == H.HGS_ERR_INVALID
    for ok in (H.make_config(rect_mode=2), H.make_config(batch=224)):
        assert L.hgs_layout(cams, 1, ctypes.byref(ok), None, None) == H.HGS_OK
    bad_mip = H.make_config()
    bad_mip.mip = 2
    assert L.hgs_layout(cams, 1, ctypes.byref(bad_mip), None, None) == H.HGS_ERR_INVALID
    cfg = H.make_config()
    assert L.hgs_layout(cams, 0, ctypes.byref(cfg), None, None) == H.HGS_ERR_INVALID
    assert L.hgs_layout(cams, H.HGS_MAX_VIEWS + 1, ctypes.byref(cfg), None, None) == H.HGS_ERR_INVALID
    zero = H.make_cameras([scenes.identity_camera(0, 64, 64.0)])
    assert L.hgs_layout(zero, 1, ctypes.byref(cfg), None, None) == H.HGS_ERR_INVALID
    # null parameter pointers with n > 0, and an SH degree above 3
    g = H.HgsGaussians()
    g.n, g.sh_degree = 10, 0
    proj = H.HgsProj()
    st = L.hgs_project(ctypes.byref(g), cams, ctypes.c_void_p(16), 1, ctypes.byref(cfg), ctypes.byref(proj),
                       None, None)
    assert st == H.HGS_ERR_INVALID
    g.n, g.sh_degree = 0, 4
    st = L.hgs_project(ctypes.byref(g), cams, ctypes.c_void_p(16), 1, ctypes.byref(cfg), ctypes.byref(proj),
                       None, None)
    assert st == H.HGS_ERR_INVALID
    # a workspace that is too small is a capacity error, reported before any launch
    p = H.HgsProj()
    p.rec = p.depth = p.rect = p.tiles = ctypes.c_void_p(256)
    st = L.hgs_bin(ctypes.byref(p), 10, cams, 1, ctypes.byref(cfg), ctypes.c_void_p(256), 16, 1000,
                   ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256),
                   None, None)
    assert st == H.HGS_ERR_CAPACITY
    st = L.hgs_bin(ctypes.byref(p), 10, cams, 1, ctypes.byref(cfg), ctypes.c_void_p(256), 1 << 40,
                   H.HGS_MAX_PAIRS + 1, ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256),
                   ctypes.c_void_p(256), None, None)
    assert st == H.HGS_ERR_INVALID
    # projection without its FP64 scratch list
    g.n, g.sh_degree = 10, 0
    g.means = g.scales = g.quats = g.normals = g.opac1 = g.opac2 = g.sh = ctypes.c_void_p(256)
    st = L.hgs_project(ctypes.byref(g), cams, ctypes.c_void_p(16), 1, ctypes.byref(cfg), ctypes.byref(p),
                       None, None)
    assert st == H.HGS_ERR_INVALID
    # misaligned record buffer
    p.fp64_list = ctypes.c_void_p(256)
    p.rec = ctypes.c_void_p(260)
    st = L.hgs_project(ctypes.byref(g), cams, ctypes.c_void_p(16), 1, ctypes.byref(cfg), ctypes.byref(p),
                       None, None)
    assert st == H.HGS_ERR_INVALID


def test_camera_struct_layout_matches_header():
    assert ctypes.sizeof(H.HgsCamera) == 4 * (12 + 4 + 2 + 1 + 3)
    assert ctypes.sizeof(H.HgsConfig) == 10 * 4
    cams = H.make_cameras([scenes.config3_camera()])
    assert cams[0].width == 1920 and cams[0].viewmat[11] == np.float32(12.0)
