"""Host logic of the benchmark's roofline accounting, on CPU.

The bench line reports every phase of the step against its roofline: the blends by their FP32
work per visited (pixel, Gaussian) position, the other phases by the bytes they must move at
least. These tests recompute the models by hand for a small made-up step, check the tile count
of ceil-divided views, and check that the traffic table's rows are read back as written.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Workload:
    def __init__(self, cameras):
        self.cameras = cameras


def test_views_tiles_rounds_partial_tiles_up():
    wl = _Workload([{"width": 1920, "height": 1080}, {"width": 640, "height": 480},
                    {"width": 17, "height": 1}])
    tuned = {"tile_w": 16, "tile_h": 16}
    # 120 x 68, 40 x 30, 2 x 1 tiles
    assert bench.views_tiles(wl, tuned) == 120 * 68 + 40 * 30 + 2


def test_phase_models_match_hand_counts():
    n, V, K, tiles = 1000, 4, 16, 300
    stats = {"n_visible": 2500, "n_pairs": 40_000, "n_eval": 3_000_000}
    phases = {"preprocess": 0.010, "compact": 0.002, "depth_sort": 0.004, "offsets": 0.001,
              "duplicate": 0.003, "tile_sort": 0.005, "ranges": 0.001,
              "blend_forward": 0.020, "blend_backward": 0.030, "preprocess_backward": 0.004,
              "unused": 0.0}
    hbm, fp32 = 5000.0, 80.0
    out = bench.phase_rooflines(phases, stats, n, V, K, tiles, hbm, fp32)
    assert "unused" not in out  # phases that did not run are left out
    nv, P = 2500, 40_000
    tile_bits = int(np.ceil(np.log2(tiles + 2)))  # ids 0 .. tiles (tiles marks an unused slot)
    expect_bytes = {
        "preprocess": 44 * n + n * V / 8 + nv * (44 + 12 * K + 52),
        "compact": n * V / 8 + 28 * nv,
        "depth_sort": 80 * nv,
        "offsets": 8 * nv,
        "duplicate": 8 * P + 44 * nv,
        "tile_sort": -(-tile_bits // 8) * 20 * P,  # under 4M pairs: 8-bit passes
        "ranges": 4 * P + 32 * tiles,
        "preprocess_backward": 128 * nv + 8 * (11 + 3 * K) * n,
    }
    for name, b in expect_bytes.items():
        r = out[name]
        assert r["bound"] == "hbm" and r["unit"] == "GB/s"
        assert r["bytes"] == pytest.approx(b)
        assert r["achieved"] == pytest.approx(b / (phases[name] * 1e-3) / 1e9)
        assert r["frac"] == pytest.approx(r["achieved"] / hbm)
    for name, flop in (("blend_forward", 15), ("blend_backward", 40)):
        r = out[name]
        assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
        assert r["flop"] == flop * 3_000_000
        assert r["frac"] == pytest.approx(flop * 3e6 / (phases[name] * 1e-3) / 1e12 / fp32)


def test_tile_sort_passes_follow_the_key_width_and_the_sort_path():
    # 155M pairs take the wide passes: 130,560 tiles need 17-bit keys, two 9-bit passes, and 300
    # tiles 9 bits, one pass. 1000 pairs take 8-bit passes: 3 and 2.
    many = {"n_visible": 1, "n_pairs": 155_000_000, "n_eval": 0}
    few = {"n_visible": 1, "n_pairs": 1000, "n_eval": 0}
    for stats, tiles, passes in ((many, 130_560, 2), (many, 300, 1), (few, 130_560, 3),
                                 (few, 300, 2)):
        out = bench.phase_rooflines({"tile_sort": 1.0}, stats, 1, 1, 1, tiles, 1.0, 1.0)
        assert out["tile_sort"]["bytes"] == passes * 20 * stats["n_pairs"], (tiles, passes)


def test_traffic_table_rows_are_read_back():
    # Every data row of the committed table parses to its bytes-per-launch cell; an unknown
    # configuration reads as None.
    rows = []
    with open(bench.TRAFFIC_TABLE) as f:
        for line in f:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 4 and cells[3].isdigit():
                rows.append(cells)
    assert rows, "the traffic table holds no rows"
    for w, k, t, b, *_ in rows:
        assert bench.measured_traffic(w, k, t) == float(b)
    assert bench.measured_traffic("large", "blend_backward", "99x99x99") is None
