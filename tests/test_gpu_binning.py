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


def _uncovered_pixels(name, sample=None, eps=1e-4, seed=0):
    """Pixels that the blend's coverage test could accept but whose tile is not listed for the
    entry: for each sampled entry, every pixel whose exponent (the blend's quadratic form of
    Eq. alpha in base 2, from the GPU's own records, in float64) lies above log2(alpha_min) - eps
    must be in one of the entry's listed tiles. The FP32 exponent differs from this one by a few
    1e-6 at the boundary, so a complete list passes with a wide margin."""
    wl = synthetic.make(name)
    g = wl.gaussians.as_dict()
    n = g["means"].shape[0]
    V = len(wl.cameras)
    r, color, depth, alpha, state = gpu_forward(g, wl.cameras)
    tiles_x = [(c["width"] + 15) // 16 for c in wl.cameras]
    tiles_per_view = [tx * ((c["height"] + 15) // 16) for tx, c in zip(tiles_x, wl.cameras)]
    total_tiles = int(sum(tiles_per_view))
    vals, ranges = r.ctx.tile_lists(state, total_tiles)
    rec, ntiles = r.ctx.records(state, V * n)
    r.release(state)
    nonempty = ranges[:, 1] > ranges[:, 0]
    starts, ends = ranges[nonempty, 0].astype(np.int64), ranges[nonempty, 1].astype(np.int64)
    tile_of = np.repeat(np.nonzero(nonempty)[0], ends - starts)
    order = np.argsort(vals, kind="stable")
    s_vals, s_tiles = vals[order], tile_of[order]
    entries = np.nonzero(ntiles > 0)[0]
    if sample is not None and entries.size > sample:
        entries = np.sort(np.random.default_rng(seed).choice(entries, sample, replace=False))
    lo = np.searchsorted(s_vals, entries, "left")
    hi = np.searchsorted(s_vals, entries, "right")
    view_base = np.concatenate([[0], np.cumsum(tiles_per_view)])
    log2_amin = np.log2(np.float64(np.float32(1.0 / 255.0)))
    missing, checked = [], 0
    for e, a, b in zip(entries, lo, hi):
        listed = set(s_tiles[a:b].tolist())
        v = int(e // n)
        W, H = int(wl.cameras[v]["width"]), int(wl.cameras[v]["height"])
        r0 = rec[e].astype(np.float64)
        mx, my = r0[0] + r0[2], r0[1] + r0[3]
        l11, l21, l22, l2o = r0[4], r0[5], r0[6], r0[7]
        # Pixels with (l11 dx + l21 dy)^2 + (l22 dy)^2 <= k, i.e. A dx^2 + B dx dy + C dy^2 <= k.
        A, B, C, k = l11 * l11, 2.0 * l11 * l21, l21 * l21 + l22 * l22, l2o - (log2_amin - eps)
        det = 4.0 * A * C - B * B
        if k < 0 or not (A > 0 and det > 0):
            continue
        ry = np.sqrt(4.0 * A * k / det)
        ys = np.arange(max(0, int(np.ceil(my - ry))), min(H - 1, int(np.floor(my + ry))) + 1)
        if ys.size == 0:
            continue
        dy = ys - my
        disc = (B * dy) ** 2 - 4.0 * A * (C * dy * dy - k)
        ok = disc >= 0
        sq = np.sqrt(np.maximum(disc, 0.0))
        xl = np.maximum(np.ceil(mx + (-B * dy - sq) / (2 * A)), 0).astype(np.int64)
        xr = np.minimum(np.floor(mx + (-B * dy + sq) / (2 * A)), W - 1).astype(np.int64)
        for y, l, rr, good in zip(ys, xl, xr, ok):
            if not good or l > rr:
                continue
            for tx in range(l // 16, rr // 16 + 1):
                checked += 1
                t = int(view_base[v] + (y // 16) * tiles_x[v] + tx)
                if t not in listed:
                    missing.append((int(e), int(y), int(tx)))
    return missing, checked


@pytest.mark.parametrize("name,sample", [("tiny", None), ("tum", 3000)])
def test_tile_lists_hold_every_pixel_the_blend_can_cover(name, sample):
    missing, checked = _uncovered_pixels(name, sample)
    assert checked > 1000
    assert not missing, missing[:10]
