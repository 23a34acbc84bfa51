"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI on a workload,
run the oracle on the same inputs, and compare with the stated tolerances:
  colour and accumulated opacity: max-abs 1e-4; depth: relative 1e-4;
  every gradient tensor: relative L2 1e-3.
Pixels the oracle flags as ambiguous (a discrete decision within FP32 rounding of its threshold)
are left out of the forward comparison and get zero upstream gradient in the backward one.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2601_00705_gb300 import binding
from paper_2601_00705_gb300.render import Renderer

COLOR_ATOL = 1e-4
DEPTH_RTOL = 1e-4
GRAD_REL_L2 = 1e-3

_renderers = {}


def renderer(**cfg) -> Renderer:
    key = tuple(sorted(cfg.items()))
    if key not in _renderers:
        _renderers[key] = Renderer(0, **cfg)
    return _renderers[key]


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def gpu_forward(g, cams, state=0, **cfg):
    r = renderer(**cfg)
    color, depth, alpha, state = r.forward_raw(to_dev(g["means"]), to_dev(g["log_scales"]),
                                               to_dev(g["quats"]), to_dev(g["opacity_logits"]),
                                               to_dev(g["sh"]), cams, state=state)
    torch.cuda.synchronize()
    return r, color, depth, alpha, state


def gpu_render(g, cams, d_color=None, d_depth=None, d_alpha=None, grad_mask=binding.GRAD_ALL,
               **cfg):
    r, color, depth, alpha, state = gpu_forward(g, cams, **cfg)
    out = dict(color=color.cpu().numpy().astype(np.float64),
               depth=depth.cpu().numpy().astype(np.float64),
               alpha=alpha.cpu().numpy().astype(np.float64))
    out["stats"] = r.stats(state)
    # No overflow (bits 1, 2) and no abandoned wait in a single-pass scan (bit 4).
    assert out["stats"]["status"] == 0, out["stats"]
    if d_color is not None or d_depth is not None or d_alpha is not None:
        n = g["means"].shape[0]
        K = g["sh"].shape[1]
        grads = r.backward_raw(state, n, K, len(cams),
                               to_dev(d_color) if d_color is not None else None,
                               to_dev(d_depth) if d_depth is not None else None,
                               to_dev(d_alpha) if d_alpha is not None else None, grad_mask)
        torch.cuda.synchronize()
        for k, v in grads.items():
            out["g_" + k] = None if v is None else v.cpu().numpy().astype(np.float64)
    r.release(state)
    return out


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))


# Largest fraction of the compared pixels the oracle may flag as ambiguous (a discrete decision
# within the modelled FP32 error of its threshold) per workload: about twice the fraction
# measured on the tests' inputs (tiny 1.6e-4, replica and tum 5.5e-4, uneven 6.5e-4, large
# 2.9e-3). A larger fraction means the flag model or its margins widened.
AMBIGUOUS_BUDGET = dict(tiny=4e-4, replica=1.2e-3, tum=1.2e-3, uneven=1.3e-3, large=6e-3)


def compare_forward(gpu, orc, mask=None, budget=None):
    """Asserts forward parity on non-ambiguous pixels, and that at most `budget` of the compared
    pixels are ambiguous; returns a dict of the measured errors."""
    ok = (orc["ambiguous"] & oracle.FORWARD_AMBIGUOUS) == 0
    if mask is not None:
        ok &= mask
    ec = np.abs(gpu["color"] - orc["color"])[ok].max(initial=0.0)
    ea = np.abs(gpu["alpha"] - orc["alpha"])[ok].max(initial=0.0)
    ed = (np.abs(gpu["depth"] - orc["depth"]) / np.maximum(np.abs(orc["depth"]), 1e-2))[ok]
    ed = ed.max(initial=0.0)
    info = dict(color_max_abs=float(ec), alpha_max_abs=float(ea), depth_max_rel=float(ed),
                ambiguous_fraction=float(1.0 - ok.mean()) if mask is None else
                float(1.0 - ok[mask].mean()))
    # Pixels whose propagated FP32 error bound is large (no discrete decision near a threshold):
    # compared like the others above, and their largest errors reported separately.
    cond = ok & ((orc["ambiguous"] & oracle.AMB_COND) != 0)
    if cond.any():
        info["cond_fraction"] = float(cond.mean() if mask is None else cond[mask].mean())
        info["cond_color_max_abs"] = float(np.abs(gpu["color"] - orc["color"])[cond].max())
        info["cond_alpha_max_abs"] = float(np.abs(gpu["alpha"] - orc["alpha"])[cond].max())
    assert ec <= COLOR_ATOL, info
    assert ea <= COLOR_ATOL, info
    assert ed <= DEPTH_RTOL, info
    if budget is not None:
        assert info["ambiguous_fraction"] <= budget, info
    return info


GRAD_KEYS = ("g_means", "g_log_scales", "g_quats", "g_opacity_logits", "g_sh", "g_pose")


def compare_backward(gpu, orc, keys=GRAD_KEYS):
    errs = {}
    for k in keys:
        if gpu.get(k) is None:
            continue
        errs[k] = rel_l2(gpu[k], orc[k])
    bad = {k: e for k, e in errs.items() if not e <= GRAD_REL_L2}
    assert not bad, errs
    return errs


def masked_l1_upstream(orc, target, weight=1.0, mask=None, eps=1e-3):
    """Upstream gradient of weight * mean L1 (oracle render vs target), zero on pixels the oracle
    flags (any decision or kink near its threshold) and where the residual is within eps."""
    P = orc["color"].shape[0]
    res = orc["color"] - target
    g = weight * np.sign(res) / P
    keep = (orc["ambiguous"] & oracle.BACKWARD_AMBIGUOUS) == 0
    if mask is not None:
        keep &= mask
    g[np.abs(res) < eps] = 0.0
    g[~keep] = 0.0
    return g.astype(np.float32), keep
