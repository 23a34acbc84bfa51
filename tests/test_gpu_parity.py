"""GPU parity: the sm_103a library, called through its C ABI, against the FP64 oracle.

Primitive kernels are checked bit-exactly (scan vs numpy cumsum, radix sort vs numpy's stable
argsort); renders and gradients within the stated tolerances (colour / opacity max-abs 1e-4,
depth relative 1e-4, gradients relative L2 1e-3) on seeded synthetic workloads.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_00705_gb300 import binding, synthetic

from gpu_common import (AMBIGUOUS_BUDGET, compare_backward, compare_forward, gpu_render,
                        masked_l1_upstream, renderer, to_dev)

pytestmark = pytest.mark.gpu


def _ctx():
    return renderer().ctx


# Up to 64k elements the scan is one cluster launch, above it three kernels: both are covered.
@pytest.mark.parametrize("n", [1, 31, 4095, 4096, 4097, 65536, 65537, 1_000_003])
def test_exclusive_scan_matches_cumsum(n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 1000, size=n).astype(np.uint32)
    xin = torch.from_numpy(x.view(np.int32)).cuda()
    out = torch.empty_like(xin)
    tot = torch.zeros(1, dtype=torch.int32, device="cuda")
    _ctx().exclusive_scan_u32(xin.data_ptr(), out.data_ptr(), n, tot.data_ptr())
    exp = np.concatenate([[0], np.cumsum(x.astype(np.uint64))[:-1]]).astype(np.uint32)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), exp)
    assert int(tot.item()) == int(x.astype(np.uint64).sum())


# Sizes up to 56 * 1024 = 57344 run as one cluster launch (16- or 8-block clusters), larger ones
# as three kernels per pass; both are covered, including the boundary and slices that leave the
# last blocks of the cluster empty.
@pytest.mark.parametrize("n,begin,end,distinct", [
    (1, 0, 32, 10), (17, 0, 31, 3), (1000, 0, 8, 7), (4096, 0, 14, 300), (4097, 3, 17, 50),
    (30_000, 0, 31, 40), (57_344, 5, 29, 1 << 29), (57_345, 0, 24, 1 << 12),
    (100_000, 0, 31, 1 << 30), (100_000, 0, 31, 50), (250_001, 0, 20, 5000),
    (1_000_000, 0, 32, 1 << 32)])
def test_radix_sort_is_stable_and_matches_numpy(n, begin, end, distinct):
    rng = np.random.default_rng(n + begin)
    keys = rng.integers(0, distinct, size=n, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    k = torch.from_numpy(keys.view(np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    _ctx().radix_sort_u32(k.data_ptr(), v.data_ptr(), n, begin, end)
    mask = np.uint64((1 << (end - begin)) - 1)
    digits = (keys.astype(np.uint64) >> np.uint64(begin)) & mask
    order = np.argsort(digits, kind="stable")
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint32), keys[order])
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), vals[order])


# From 4M keys (capacity) the sort takes passes of up to 9 bits in blocks of 8192 keys.
@pytest.mark.parametrize("n,begin,end,runs", [
    (4_194_304, 0, 17, False), (4_194_305, 0, 17, True), (5_000_003, 0, 32, False),
    (9_000_001, 3, 20, True), (8_191 * 1024 + 7, 0, 31, True)])
def test_wide_radix_sort_is_stable_and_matches_numpy(n, begin, end, runs):
    rng = np.random.default_rng(n + begin)
    if runs:
        # Pair-list-like keys: runs of consecutive values (a footprint's tiles), runs in random
        # order, so that a warp's keys share their high digits.
        starts = rng.integers(0, 1 << min(end, 31), size=n // 6 + 1, dtype=np.uint64)
        keys = (starts[:, None] + np.arange(6, dtype=np.uint64)[None, :]).ravel()[:n]
        keys = (keys % np.uint64(1 << 32)).astype(np.uint32)
    else:
        keys = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    k = torch.from_numpy(keys.view(np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    _ctx().radix_sort_u32(k.data_ptr(), v.data_ptr(), n, begin, end)
    mask = np.uint64((1 << (end - begin)) - 1)
    digits = (keys.astype(np.uint64) >> np.uint64(begin)) & mask
    order = np.argsort(digits, kind="stable")
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint32), keys[order])
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), vals[order])


def test_radix_sort_keys_only():
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 1 << 31, size=123_457, dtype=np.uint64).astype(np.uint32)
    k = torch.from_numpy(keys.view(np.int32)).cuda()
    _ctx().radix_sort_u32(k.data_ptr(), 0, keys.size, 0, 32)
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint32), np.sort(keys))


# ----------------------------------------------------------------------------- renders

def _oracle_l1_case(wl, seed=2001, weight_depth=0.0, mask=None):
    g = wl.gaussians.as_dict()
    orc0 = oracle.render(g, wl.cameras)
    rng = np.random.default_rng(seed)
    target = rng.random(orc0["color"].shape)
    d_color, keep = masked_l1_upstream(orc0, target, mask=mask)
    d_depth = None
    if weight_depth:
        tdepth = orc0["depth"] * rng.uniform(0.9, 1.1, size=orc0["depth"].shape)
        res = orc0["depth"] - tdepth
        d_depth = (weight_depth * np.sign(res) / res.size).astype(np.float32)
        d_depth[(np.abs(res) < 1e-4) | ~keep] = 0.0
    return g, orc0, d_color, d_depth


def test_tiny_forward_and_all_gradients():
    wl = synthetic.tiny()
    g, orc0, d_color, _ = _oracle_l1_case(wl)
    d_alpha = (np.random.default_rng(5).standard_normal(orc0["alpha"].shape) * 1e-4).astype(np.float32)
    keep = (orc0["ambiguous"] & oracle.BACKWARD_AMBIGUOUS) == 0
    d_alpha[~keep] = 0.0
    orc = oracle.render(g, wl.cameras, d_color=d_color, d_alpha=d_alpha)
    gpu = gpu_render(g, wl.cameras, d_color=d_color, d_alpha=d_alpha)
    info = compare_forward(gpu, orc, budget=AMBIGUOUS_BUDGET["tiny"])
    errs = compare_backward(gpu, orc)
    print("tiny", info, errs, gpu["stats"])


def _assert_same_forward(out, ref, orc, same_tile_shape):
    """Per-pixel compositing does not depend on the binning. Within one tile shape every pixel's
    exponent is formed from the same tile anchor row whatever the pixels per thread, so the
    forward is bit-identical; another tile shape rounds the whitened offsets from another anchor
    row, which moves values by float32 rounding only (decisions the oracle flags as within that
    rounding of their threshold may go either way there)."""
    if same_tile_shape:
        for k in ("color", "depth", "alpha"):
            np.testing.assert_array_equal(out[k], ref[k], err_msg=k)
        return
    ok = (orc["ambiguous"] & oracle.FORWARD_AMBIGUOUS) == 0
    for k in ("color", "depth", "alpha"):
        np.testing.assert_allclose(out[k][ok], ref[k][ok], rtol=0, atol=1e-5, err_msg=k)


@pytest.mark.parametrize("tile", [(16, 16, 1), (16, 16, 2), (16, 16, 8), (8, 8, 1), (8, 8, 2),
                                  (32, 8, 1), (32, 8, 2), (32, 8, 4), (32, 8, 8),
                                  (16, 16, 8, 2), (16, 16, 1, 8), (32, 8, 2, 8), (8, 8, 2, 1)])
def test_tile_shape_and_pixels_per_thread_do_not_change_results(tile):
    """tile = (tile_w, tile_h, pixels per thread[, backward pixels per thread])."""
    wl = synthetic.tiny(seed=77)
    g, orc0, d_color, _ = _oracle_l1_case(wl)
    ref = gpu_render(g, wl.cameras, d_color=d_color)  # default: 16x16 tiles, 4 pixels per thread
    out = gpu_render(g, wl.cameras, d_color=d_color, tile_w=tile[0], tile_h=tile[1],
                     pixels_per_thread=tile[2],
                     backward_pixels_per_thread=tile[3] if len(tile) > 3 else 0)
    _assert_same_forward(out, ref, orc0, same_tile_shape=tile[:2] == (16, 16))
    for k in ("g_means", "g_log_scales", "g_quats", "g_opacity_logits", "g_sh", "g_pose"):
        np.testing.assert_allclose(out[k], ref[k], rtol=1e-4, atol=1e-6 * np.abs(ref[k]).max(),
                                   err_msg=k)


@pytest.mark.parametrize("bwd_ppt,weight_depth", [(8, 0.0), (4, 0.0), (1, 0.0), (8, 0.1)])
def test_long_tile_runs_backward_matches_oracle(bwd_ppt, weight_depth):
    """Runs of thousands of Gaussians per tile (the crowded scene: its longest run exceeds 8192,
    see the binning test, and most depths are shared by ~30 Gaussians): the backward walks many
    staged batches and reduction groups per tile; every gradient against the oracle, for one,
    two and eight warps per tile; with a depth term in the loss, the blend's depth variant."""
    wl = synthetic.crowded()
    g, orc0, d_color, d_depth = _oracle_l1_case(wl, weight_depth=weight_depth)
    orc = oracle.render(g, wl.cameras, d_color=d_color, d_depth=d_depth)
    gpu = gpu_render(g, wl.cameras, d_color=d_color, d_depth=d_depth, tile_w=16, tile_h=16,
                     pixels_per_thread=4, backward_pixels_per_thread=bwd_ppt)
    assert gpu["stats"]["n_pairs"] > 2 * 8192
    info = compare_forward(gpu, orc)
    errs = compare_backward(gpu, orc)
    print("crowded", bwd_ppt, weight_depth, info, errs)


def test_replica_forward_and_pose_gradient():
    wl = synthetic.replica()
    g, orc0, d_color, d_depth = _oracle_l1_case(wl, weight_depth=0.1)
    orc = oracle.render(g, wl.cameras, d_color=d_color, d_depth=d_depth)
    gpu = gpu_render(g, wl.cameras, d_color=d_color, d_depth=d_depth, grad_mask=binding.GRAD_POSE)
    info = compare_forward(gpu, orc, budget=AMBIGUOUS_BUDGET["replica"])
    errs = compare_backward(gpu, orc, keys=("g_pose",))
    print("replica", info, errs, gpu["stats"])


@pytest.mark.slow
def test_tum_window_all_gradients():
    wl = synthetic.tum()
    g, orc0, d_color, _ = _oracle_l1_case(wl)
    orc = oracle.render(g, wl.cameras, d_color=d_color)
    gpu = gpu_render(g, wl.cameras, d_color=d_color)
    info = compare_forward(gpu, orc, budget=AMBIGUOUS_BUDGET["tum"])
    errs = compare_backward(gpu, orc)
    print("tum", info, errs, gpu["stats"])


# ----------------------------------------------------------------------------- edge cases

def test_empty_scene_renders_background():
    wl = synthetic.tiny(n=0)
    g = wl.gaussians.as_dict()
    bg = (0.25, 0.5, 0.75)
    P = wl.n_pixels
    gpu = gpu_render(g, wl.cameras, d_color=np.ones((P, 3), np.float32), bg=bg)
    np.testing.assert_array_equal(gpu["alpha"], 0.0)
    np.testing.assert_array_equal(gpu["depth"], 0.0)
    np.testing.assert_allclose(gpu["color"], np.tile(np.float32(bg), (P, 1)), rtol=0, atol=0)
    np.testing.assert_array_equal(gpu["g_pose"], 0.0)


def test_everything_behind_the_near_plane():
    wl = synthetic.tiny(n=500)
    g = dict(wl.gaussians.as_dict())
    g["means"] = g["means"].copy()
    g["means"][:, 2] = 0.1  # z <= znear = 0.2
    P = wl.n_pixels
    gpu = gpu_render(g, wl.cameras, d_color=np.ones((P, 3), np.float32))
    assert gpu["stats"]["n_visible"] == 0
    np.testing.assert_array_equal(gpu["alpha"], 0.0)
    for k in ("g_means", "g_sh", "g_pose"):
        np.testing.assert_array_equal(gpu[k], 0.0)


def test_nonfinite_gaussians_are_culled_and_counted():
    wl = synthetic.tiny(n=300)
    g = {k: v.copy() for k, v in wl.gaussians.as_dict().items()}
    # Three Gaussians that the view sees, each with one non-finite parameter.
    proj = oracle.project(g, wl.cameras)
    m2 = proj["mean2d"][0]
    on = np.nonzero(proj["valid"][0] & (m2[:, 0] > 10) & (m2[:, 0] < 150) & (m2[:, 1] > 10) &
                    (m2[:, 1] < 110))[0]
    bad = [int(on[3]), int(on[10]), int(on[20])]
    g["means"][bad[0], 0] = np.nan
    g["log_scales"][bad[1], 1] = np.inf
    g["sh"][bad[2], 0, 2] = -np.inf
    gpu = gpu_render(g, wl.cameras, d_color=np.ones((wl.n_pixels, 3), np.float32) / wl.n_pixels)
    assert gpu["stats"]["n_nonfinite"] == 3
    for k in ("color", "alpha", "depth", "g_means", "g_sh", "g_pose"):
        assert np.isfinite(gpu[k]).all(), k
    for i in bad:
        assert not gpu["g_means"][i].any()
    # The remaining Gaussians render exactly as without the three bad ones.
    keep = np.setdiff1d(np.arange(300), bad)
    g2 = {k: v[keep] for k, v in g.items()}
    ref = gpu_render(g2, wl.cameras)
    np.testing.assert_allclose(gpu["color"], ref["color"], atol=1e-6)


def test_autotuner_choice_is_valid_cached_and_leaves_results_unchanged():
    from paper_2601_00705_gb300.render import Renderer
    wl = synthetic.tiny(seed=3)
    g = wl.gaussians.as_dict()
    r = Renderer(0)
    params = [to_dev(g[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    first = r.autotune(*params, wl.cameras)
    assert (first["tile_w"], first["tile_h"]) in {(16, 16), (8, 8), (32, 8)}
    assert first["pixels_per_thread"] in (1, 2, 4, 8) and first["ms"] > 0
    assert first["backward_pixels_per_thread"] in (1, 2, 4, 8)
    for k in ("pixels_per_thread", "backward_pixels_per_thread"):
        assert first["tile_w"] * first["tile_h"] // first[k] % 32 == 0
    keys = ("tile_w", "tile_h", "pixels_per_thread", "backward_pixels_per_thread")
    second = r.autotune(*params, wl.cameras)
    assert second["ms"] == 0 and {k: second[k] for k in keys} == {k: first[k] for k in keys}
    tuned = gpu_render(g, wl.cameras, tile_w=first["tile_w"], tile_h=first["tile_h"],
                       pixels_per_thread=first["pixels_per_thread"],
                       backward_pixels_per_thread=first["backward_pixels_per_thread"])
    ref = gpu_render(g, wl.cameras)
    _assert_same_forward(tuned, ref, oracle.render(g, wl.cameras),
                         same_tile_shape=(first["tile_w"], first["tile_h"]) == (16, 16))
