"""Invariants of the binning stage on the GPU (tile scan, scatter, per-tile depth sort), checked
on the library's own sorted pair lists:
  * the tile ranges partition the pair list in tile order;
  * every tile's run is strictly increasing in (float32 depth, Gaussian index), i.e. the
    near-to-far order of Section 3.2.2 with ties by index, and holds each Gaussian at most once;
  * a (view, Gaussian) entry appears in exactly as many tiles as its tile count, all in its own
    view.
"""
import numpy as np
import pytest

from paper_2601_00705_gb300 import synthetic

import oracle

from gpu_common import compare_forward, gpu_forward, gpu_render

pytestmark = pytest.mark.gpu


def _check_lists(name, **kw):
    wl = synthetic.make(name, **kw)
    g = wl.gaussians.as_dict()
    n = g["means"].shape[0]
    V = len(wl.cameras)
    r, color, depth, alpha, state = gpu_forward(g, wl.cameras)
    tiles_per_view = [((c["width"] + 15) // 16) * ((c["height"] + 15) // 16) for c in wl.cameras]
    total_tiles = int(sum(tiles_per_view))
    vals, ranges = r.ctx.tile_lists(state, total_tiles)
    rec, ntiles = r.ctx.records(state, V * n)
    r.release(state)
    P = vals.size
    max_run = int((ranges[:, 1].astype(np.int64) - ranges[:, 0]).max()) if P else 0
    assert P == int(ntiles.astype(np.int64).sum())
    # Ranges partition [0, P) in tile order (empty tiles are [0, 0)).
    nonempty = ranges[:, 1] > ranges[:, 0]
    starts, ends = ranges[nonempty, 0].astype(np.int64), ranges[nonempty, 1].astype(np.int64)
    assert starts[0] == 0 and ends[-1] == P
    np.testing.assert_array_equal(starts[1:], ends[:-1])
    # Each pair's tile and view.
    tile_of = np.repeat(np.nonzero(nonempty)[0], ends - starts)
    view_base = np.concatenate([[0], np.cumsum(tiles_per_view)])
    view_of_tile = np.searchsorted(view_base, tile_of, side="right") - 1
    np.testing.assert_array_equal(vals // n, view_of_tile)
    # Strict (depth bits, index) order inside every run.
    zbits = rec[vals, 11].view(np.uint32).astype(np.uint64)
    key = (zbits << np.uint64(32)) | (vals % n).astype(np.uint64)
    same_tile = tile_of[1:] == tile_of[:-1]
    bad = np.nonzero(same_tile & (key[1:] <= key[:-1]))[0]
    assert bad.size == 0, (name, bad[:10], tile_of[bad[:10]], vals[bad[:10]], vals[bad[:10] + 1])
    # Every entry appears in exactly ntiles of its view's tiles.
    counts = np.bincount(vals, minlength=V * n)
    np.testing.assert_array_equal(counts, ntiles)
    return max_run


@pytest.mark.parametrize("name,kw", [("tiny", {}), ("tum", {}), ("uneven", {})])
def test_tile_lists_are_ordered_and_complete(name, kw):
    _check_lists(name, **kw)


@pytest.mark.slow
def test_tile_lists_are_ordered_and_complete_large():
    _check_lists("large")


def test_long_tile_runs_are_merged_in_order_with_depth_ties():
    # Runs longer than one shared-memory sort block (2048 keys) are sorted block by block and
    # merged; most depths are shared by ~30 Gaussians, so the index tie-break decides often.
    max_run = _check_lists("crowded")
    assert max_run > 4 * 2048, max_run
    wl = synthetic.crowded()
    g = wl.gaussians.as_dict()
    orc = oracle.render(g, wl.cameras)
    gpu = gpu_render(g, wl.cameras)
    print("crowded", max_run, compare_forward(gpu, orc), gpu["stats"])
