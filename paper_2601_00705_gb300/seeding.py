"""Dense initialisation of Gaussian seeds from matched keyframe pixels (Section 3.3 "Multi-view
Triangulation" and "Gaussian Parameter Initialization"; appendix Eq. app-sigma-init,
Eq. app-alpha-init), on the device through the C ABI.

``triangulate`` runs the FP64 two-view DLT per (reference pixel, neighbour) and keeps the best
accepted hypothesis per pixel; ``init_seeds`` turns the accepted points into Gaussian parameters
in the renderer's layout (means, log-scales, quaternions, opacity logits, SH), plus normals.
"""
from __future__ import annotations

import torch

from . import binding


def _dev(t, dtype, device):
    return torch.as_tensor(t).to(device=device, dtype=dtype).contiguous()


def triangulate(ctx: binding.Context, cameras, ref_view, ref_xy, nb_view, nb_xy, nb_conf,
                device, stream: int = 0, **config) -> dict:
    """Inputs (host or device): ref_view [M], ref_xy [M,2], nb_view [M,K] (-1: none),
    nb_xy [M,K,2], nb_conf [M,K]. Returns device tensors valid [M] (bool), X [M,3] (float64),
    best [M], err [M], angle [M], kappa [M], and the inputs as device tensors (key "inputs")."""
    rv = _dev(ref_view, torch.int32, device)
    M = int(rv.shape[0])
    K = int(torch.as_tensor(nb_view).shape[-1])
    nv = _dev(nb_view, torch.int32, device).reshape(M, K)
    inp = dict(ref_view=rv, ref_xy=_dev(ref_xy, torch.float64, device).reshape(M, 2),
               nb_view=nv, nb_xy=_dev(nb_xy, torch.float64, device).reshape(M, K, 2),
               nb_conf=_dev(nb_conf, torch.float32, device).reshape(M, K))
    out = dict(valid=torch.empty(M, dtype=torch.int32, device=device),
               X=torch.empty((M, 3), dtype=torch.float64, device=device),
               best=torch.empty(M, dtype=torch.int32, device=device),
               err=torch.empty(M, dtype=torch.float64, device=device),
               angle=torch.empty(M, dtype=torch.float64, device=device),
               kappa=torch.empty(M, dtype=torch.float32, device=device))
    ptrs = {k: v.data_ptr() for k, v in {**inp, **out}.items()}
    ctx.triangulate(binding.make_cameras(cameras), M, K, ptrs,
                    binding.default_seed_config(**config), stream)
    out["inputs"] = inp
    return out


def init_seeds(ctx: binding.Context, cameras, tri: dict, observed, gain_bias, device,
               sh_degree: int = 0, stream: int = 0, **config) -> dict:
    """Seeds of the accepted points of ``triangulate`` (its output dict). Returns device tensors
    index [S], means [S,3], log_scales [S,3], quats [S,4], opacity_logits [S], sh [S,K,3],
    normals [S,3]."""
    inp = tri["inputs"]
    M, K = inp["nb_view"].shape
    Ksh = (sh_degree + 1) ** 2
    f32 = dict(dtype=torch.float32, device=device)
    out = dict(index=torch.empty(M, dtype=torch.int32, device=device),
               means=torch.empty((M, 3), **f32), log_scales=torch.empty((M, 3), **f32),
               quats=torch.empty((M, 4), **f32), opacity_logits=torch.empty(M, **f32),
               sh=torch.empty((M, Ksh, 3), **f32), normals=torch.empty((M, 3), **f32))
    obs = _dev(observed, torch.float32, device)
    gb = _dev(gain_bias, torch.float32, device)
    ptrs = dict(ref_view=inp["ref_view"].data_ptr(), nb_view=inp["nb_view"].data_ptr(),
                valid=tri["valid"].data_ptr(), X=tri["X"].data_ptr(), err=tri["err"].data_ptr(),
                angle=tri["angle"].data_ptr(), kappa=tri["kappa"].data_ptr(),
                observed=obs.data_ptr(), gain_bias=gb.data_ptr(),
                **{k: v.data_ptr() for k, v in out.items()})
    S = ctx.init_seeds(binding.make_cameras(cameras), M, K, ptrs, sh_degree,
                       binding.default_seed_config(**config), stream)
    return {k: v[:S] for k, v in out.items()}
