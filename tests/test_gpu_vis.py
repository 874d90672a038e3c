"""The visibility mask the forward compositing writes for the backward.

For each tile, each 32-entry chunk of its sorted list and each 8x4 pixel block of
the tile, one uint32 word: bit j is set iff list entry beg + 32c + j is composited
(before the 1e-4 stop, at or above the 1/255 floor; Sec. 3.3 blending with the
Eq. 10 weight) at some pixel of the block.  The expected words come from the FP64
oracle's per-(pair, pixel) composited flags, packed by the layout include/hgs.h
states; they must equal the GPU's bit for bit in every block whose pixels FP32 can
decide as FP64 does (no exempt pixel), up to the chunk of the block's last
composited entry (later chunks are not written).  The backward visits only the
marked entries, so a second test runs it with no room for the mask (every entry
visited) and checks the gradients are the same."""
import numpy as np
import pytest

import oracle
from hgs_testutil import exempt, gpu_render, masked_upstream
from paper_2406_02720_b300 import scenes

pytestmark = pytest.mark.gpu


def _expected_words(ref, ranges_gpu, tile_ids, cam, tile):
    """{word index: expected word} from the oracle's composited flags of one view;
    ranges_gpu / tile_ids: the GPU's [start, end) and global id of each of the view's
    tiles (the list order is the oracle's, bit-exact)."""
    tw, th = tile
    nw = tw * th // 32
    tiles_x = (cam.width + tw - 1) // tw
    comp, rng_o = ref["comp"], ref["bins"]["ranges"].reshape(-1, 2)
    ex = exempt(ref)
    words = {}
    for t, (beg_o, end_o) in enumerate(rng_o):
        beg, end = (int(x) for x in ranges_gpu[t])
        assert end - beg == end_o - beg_o
        tx, ty = t % tiles_x, t // tiles_x
        for w in range(nw):
            bx, by = (w % (tw // 8)) * 8, (w // (tw // 8)) * 4       # block origin in the tile
            x0, y0 = tx * tw + bx, ty * th + by
            xs, ys = slice(x0, min(x0 + 8, cam.width)), slice(y0, min(y0 + 4, cam.height))
            if x0 >= cam.width or y0 >= cam.height or ex[ys, xs].any():
                continue
            last = int(ref["n_contrib"][ys, xs].max())
            if last == 0:
                continue
            hit = comp[beg_o:end_o, by:by + 4, bx:bx + 8].any(axis=(1, 2))
            for c in range((last - 1) // 32 + 1):
                bits = hit[32 * c:32 * c + 32]
                word = int(np.sum(bits.astype(np.uint64) << np.arange(bits.size, dtype=np.uint64)))
                words[((beg >> 5) + int(tile_ids[t]) + c) * nw + w] = word
    return words


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_mask_matches_the_oracle(cuda_ok, tile):
    rng = np.random.default_rng(43)
    sc = scenes.scene_uniform(rng, 1500, [-1.6, -1.1, 2.5], [1.6, 1.1, 6.5], -3.2, 0.6, 1.5, 2)
    cams = [scenes.identity_camera(150, 93, 85.0, 75.0, 46.5, bg=(0.1, 0.2, 0.3)),
            scenes.identity_camera(72, 40, 40.0, 36.0, 20.0)]
    out = gpu_render(sc, cams, tile=tile)
    r = out["rast"]
    assert r.read_status() == 0
    vis = r.vis.cpu().numpy().view(np.uint32)
    nw = tile[0] * tile[1] // 32
    assert vis.size == (r.capacity // 32 + r.total_tiles + 1) * nw
    toff, checked, set_bits = 0, 0, 0
    for v, cam in enumerate(cams):
        ref = oracle.render(sc, cam, tile=tile, composited=True)
        nt = ref["bins"]["ranges"].size // 2
        exp = _expected_words(ref, out["ranges"][toff:toff + nt], np.arange(toff, toff + nt), cam, tile)
        for wi, word in exp.items():
            assert vis[wi] == word, (v, wi, hex(int(vis[wi])), hex(word))
        checked += len(exp)
        set_bits += sum(bin(x).count("1") for x in exp.values())
        toff += nt
    assert checked > 50 and set_bits > 500


def test_backward_without_room_for_the_mask(cuda_ok):
    """No room for the mask: the forward reports HGS_DEV_CAPACITY and writes no word,
    the image is unchanged, and the backward (every entry visited) gives the same
    gradients as with the mask."""
    import torch
    from paper_2406_02720_b300 import hgs as H
    rng = np.random.default_rng(44)
    sc = scenes.scene_uniform(rng, 1200, [-1.5, -1.0, 2.5], [1.5, 1.0, 6.0], -3.2, 0.6, 1.5, 1)
    cams = [scenes.identity_camera(128, 80, 80.0, 64.0, 40.0)]
    ref = oracle.render(sc, cams[0])
    dL = masked_upstream(scenes.upstream_grad(102, cams), [ref])
    out = gpu_render(sc, cams, dL=dL)
    r = out["rast"]
    g_mask = r.grad2d.clone()
    img = r.image.clone()
    r.vis = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    r.clear_status()
    r.render_fwd()
    assert r.read_status() == H.HGS_DEV_CAPACITY
    assert int(r.vis.item()) == -1                     # nothing written
    assert torch.equal(r.image, img)
    r.clear_status()
    r.rasterize_bwd(torch.from_numpy(np.asarray(dL[0], np.float32).reshape(-1)).cuda())
    assert r.read_status() == 0
    a, b = g_mask.cpu().numpy(), r.grad2d.cpu().numpy()
    scale = np.abs(a).max(axis=0) + 1e-30
    np.testing.assert_allclose(b / scale, a / scale, rtol=0, atol=1e-6)
    assert np.count_nonzero(a) > 1000
