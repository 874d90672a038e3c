"""Host-side logic of bench.py, on CPU: the max-over-ranks timing and whole-job
aggregate over two gloo ranks, the launch and byte accounting, the clock summary,
and the reference arm's rank rule."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench as b
    dist = b.init_dist(ws, "gloo")
    ms = 2.0 + 3.0 * rank                               # rank 1 is the slow one
    ms_max = b.max_over_ranks(ms, dist)
    out[rank] = (ms_max, b.aggregate_value(1920 * 1080, ws, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_two_gloo_ranks():
    ws = 2
    port = 29000 + os.getpid() % 1000
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        ms_max, v = res[r]
        assert ms_max == 5.0
        assert v == pytest.approx(2 * 1920 * 1080 / 5.0e3)


def test_single_rank_needs_no_process_group():
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.aggregate_value(1e6, 1, 1.0) == pytest.approx(1000.0)


def test_launch_and_pass_accounting():
    # 1920x1080 in 16x16 tiles: 120 x 68 = 8160 tiles -> 13 bits -> 2 tile passes
    assert bench.tile_bits(8160) == 13
    assert bench.n_sort_passes(8160) == (4, 2)
    assert bench.n_sort_passes(8160, 3) == (3, 2)
    assert bench.n_sort_passes(256) == (4, 1)
    assert bench.n_sort_passes(257) == (4, 2)
    # project 2 + binning (1 + 3*4 + 3 + 3*2 + 1) + fwd + bwd + project_bwd 2
    assert bench.launches_per_step(8160, persistent=False) == 29
    # + queue count and fill before the forward (the backward reuses its queue)
    assert bench.launches_per_step(8160, persistent=True) == 31


def test_depth_sort_passes():
    """Passes over the depth keys: the drawn splats' key range (max - min + 1) in bits,
    8 bits a pass; culled splats (tiles 0) do not widen it."""
    import numpy as np
    depths = np.array([5.82, 18.0, 7.5, 1e30, -3.0], np.float32)    # last two culled
    tiles = np.array([3, 1, 2, 0, 0])
    span = int(np.float32(18.0).view(np.uint32)) - int(np.float32(5.82).view(np.uint32)) + 1
    assert span < 1 << 24
    assert bench.depth_sort_passes(depths, tiles) == 3
    assert bench.depth_sort_passes(np.array([1.0, 11.0], np.float32), np.array([1, 1])) == 4
    assert bench.depth_sort_passes(np.array([2.0, 2.0], np.float32), np.array([1, 1])) == 1
    assert bench.depth_sort_passes(depths, np.zeros(5, int)) == 0
    # the byte count follows the passes
    assert bench.alg_bytes(10, 0, 1, 4)["bin"] - bench.alg_bytes(10, 0, 1, 3)["bin"] == 10 * 20


def test_algorithmic_bytes():
    b = bench.alg_bytes(1000, 5000, 8160)
    assert b["project"] == 1000 * 340
    assert b["project_bwd"] == 1000 * 552
    assert b["bin"] == 1000 * (16 + 80 + 12 + 24) + 5000 * (8 + 40 + 4) + 8160 * 8
    # 64 views, 40k of the 64k (view, splat) entries drawn: parameters read once, entry
    # fields per entry, records per drawn entry; 308,780 tiles take three tile passes
    m = bench.alg_bytes(1000, 5000, 308780, depth_passes=3, views=64, drawn=40000)
    assert m["project"] == 1000 * 252 + 64000 * 24 + 40000 * 64
    assert m["project_bwd"] == 1000 * 504 + 64000 * 48
    assert m["bin"] == 64000 * (16 + 60 + 12 + 24) + 5000 * (8 + 60 + 4) + 308780 * 8


def test_clock_summary():
    rows = ["0, 2032, 2032, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1990, 2032, 1000.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 345, 2032, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage"]
    c = bench.summarize_clocks(rows)
    assert c["sm_max_mhz"] == 2032.0
    assert c["sm_mhz"] == pytest.approx((2032 + 1990) / 2)   # idle sample dropped
    assert c["reasons"] == ["sw_power_cap"]
    assert c["samples"] == 3
    assert bench.summarize_clocks([]) is None


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 1, "warmup": 3})()
    assert bench.run_reference(args) is None


def test_reference_arm_line_on_a_small_scene(monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    args = type("A", (), {"steps": 2, "warmup": 1, "n": 4000, "tile_w": 16, "tile_h": 16})()
    line = bench.run_reference(args)
    assert line["impl"] == "reference" and line["unit"] == "Mpixel/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_profiled_traffic_needs_the_profiled_source(tmp_path, monkeypatch):
    import hashlib
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    prof = tmp_path / "p.md"
    digest = hashlib.sha256(b"kernel v1").hexdigest()
    prof.write_text(f"# summary\n- source_sha256: {digest}\n- traffic_bytes_per_launch: 377340672\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.PROFILE_OF, "render_bwd", ("p.md", "k.cu"))
    assert bench.profiled_traffic("render_bwd") == 377340672.0
    src.write_text("kernel v2")                      # the kernel changed since the capture
    assert bench.profiled_traffic("render_bwd") is None
    assert bench.profiled_traffic("bin") is None


def test_backward_atomics_report():
    import bench
    stats = {"bwd_contrib": 1000, "bwd_atomic": 250}
    a = bench.bwd_atomics(stats, 0.5)
    assert a["vector_reductions"] == 750 and a["float_adds"] == 3000 and a["float_adds_unfolded"] == 12000
    assert a["pairs_per_lane_atomic"] == 4.0
    assert abs(a["G_float_adds_per_s"] - 3000 / 0.5e-3 / 1e9) < 1e-12
    assert abs(a["GB_reduced_per_s"] - 4 * a["G_float_adds_per_s"]) < 1e-12
