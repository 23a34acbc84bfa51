"""PyTorch front end: device tensors in, device tensors out, autograd through ``librgs.so``.

``render(...)`` is differentiable in the Gaussian parameters and in a per-view twist
xi = (rho, omega) of the left pose update T_WC <- exp(xi^) T_WC (Section 3.2.3, Eq. leftupdate).
The twist is evaluated at xi = 0: the cameras passed in are the current poses, and its gradient
is the pose gradient the tracker steps along (after a step, fold exp(xi^) into the cameras and
reset xi to zero). PyTorch only supplies device memory and the current stream; all arithmetic
runs in the library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding

_GRAD_BITS = (binding.GRAD_MEANS, binding.GRAD_SCALES, binding.GRAD_QUATS, binding.GRAD_OPACITY,
              binding.GRAD_SH, binding.GRAD_POSE)


def _check_param(t: torch.Tensor, name: str, shape_tail: tuple, device) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or t.device != device:
        raise TypeError(f"{name} must be a float32 tensor on {device}")
    if tuple(t.shape[1:]) != shape_tail:
        raise ValueError(f"{name} must have shape [N, {', '.join(map(str, shape_tail))}]")
    t = t.contiguous()
    if t.data_ptr() % 16:
        t = t.clone()
    return t


class Renderer:
    """One library context on one CUDA device, plus the renderer constants."""

    def __init__(self, device: int | torch.device = 0, **config):
        dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("the renderer runs on CUDA devices only")
        self.device = dev
        self.ctx = binding.Context(dev.index or 0)
        self.config = binding.default_config(**config)

    def stream_handle(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def forward_raw(self, means, log_scales, quats, opacity_logits, sh, cameras, state: int = 0,
                    out=None, world_to_cam: torch.Tensor | None = None,
                    sh_event: "torch.cuda.Event | None" = None):
        """Runs the forward; returns (color [P,3], depth [P], alpha [P], state handle).

        world_to_cam: optional device float32 tensor [V,12] (or [V,3,4]) of row-major [R|t]
        poses that replace the cameras' poses (read on the device, so a pose the device updates
        needs no host round trip).
        sh_event: optional recorded CUDA event after which `sh` holds its values; the forward
        then evaluates the colours after the sorts and waits for it only there, so the upload of
        the coefficients can overlap the projection and the sorts (without it the projection
        evaluates them)."""
        dev = self.device
        n = int(means.shape[0])
        K = int(sh.shape[1]) if sh.dim() == 3 else 0
        deg = int(round(K ** 0.5)) - 1
        if (deg + 1) ** 2 != K or not 0 <= deg <= 3:
            raise ValueError("sh must be [N, (d+1)^2, 3] with d in 0..3")
        means = _check_param(means, "means", (3,), dev)
        log_scales = _check_param(log_scales, "log_scales", (3,), dev)
        quats = _check_param(quats, "quats", (4,), dev)
        opacity_logits = _check_param(opacity_logits.reshape(n, 1), "opacity_logits", (1,), dev)
        sh = _check_param(sh, "sh", (K, 3), dev)
        cams = cameras if hasattr(cameras, "_type_") else binding.make_cameras(cameras)
        P = sum(int(c.width) * int(c.height) for c in cams)
        if out is None:
            color = torch.empty((P, 3), dtype=torch.float32, device=dev)
            depth = torch.empty((P,), dtype=torch.float32, device=dev)
            alpha = torch.empty((P,), dtype=torch.float32, device=dev)
        else:
            color, depth, alpha = out
        g = binding.Gaussians(n, deg, means.data_ptr(), log_scales.data_ptr(), quats.data_ptr(),
                              opacity_logits.data_ptr(), sh.data_ptr())
        imgs = binding.Images(color.data_ptr(), depth.data_ptr(), alpha.data_ptr())
        cfg = self.config
        if sh_event is not None:
            if not sh_event.cuda_event:
                raise ValueError("sh_event must have been recorded")
            cfg = binding.Config.from_buffer_copy(self.config)
            cfg.sh_ready_event = sh_event.cuda_event
        if world_to_cam is None:
            state = self.ctx.forward(g, cams, cfg, imgs, state, self.stream_handle())
        else:
            if (world_to_cam.device != dev or world_to_cam.dtype != torch.float32
                    or not world_to_cam.is_contiguous() or world_to_cam.numel() != 12 * len(cams)):
                raise ValueError("world_to_cam must be a contiguous float32 [V,12] tensor on the "
                                 "renderer's device")
            state = self.ctx.forward_posed(g, cams, world_to_cam.data_ptr(), cfg, imgs,
                                           state, self.stream_handle())
        # Keep the (possibly copied) parameter tensors alive for the backward.
        self._last_inputs = (means, log_scales, quats, opacity_logits, sh)
        return color, depth, alpha, state

    def backward_raw(self, state: int, n: int, K: int, n_views: int, d_color=None, d_depth=None,
                     d_alpha=None, grad_mask: int = binding.GRAD_ALL, out: dict | None = None,
                     reg: "binding.MapReg | None" = None):
        """Runs the backward of `state`; returns a dict of gradient tensors (None if not asked).
        `out` may supply preallocated float32 tensors (keys means, log_scales, quats,
        opacity_logits, sh, pose). `reg` adds the mapping regulariser (Eq. reg) and advances the
        maintenance counters (see ``mapping.MapRegularizer``)."""
        dev = self.device

        def prep(t, shape):
            if t is None:
                return None
            t = t.to(dtype=torch.float32).contiguous()
            return t.reshape(shape)

        d_color = prep(d_color, (-1, 3))
        d_depth = prep(d_depth, (-1,))
        d_alpha = prep(d_alpha, (-1,))
        given = out or {}
        out = {}
        shapes = dict(means=(n, 3), log_scales=(n, 3), quats=(n, 4), opacity_logits=(n,),
                      sh=(n, K, 3), pose=(n_views, 6))
        for (name, shape), bit in zip(shapes.items(), _GRAD_BITS):
            if not grad_mask & bit:
                out[name] = None
            elif given.get(name) is not None:
                t = given[name]
                if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != int(
                        np.prod(shape)) or t.data_ptr() % 16:
                    raise ValueError(f"preallocated gradient '{name}' must be a contiguous, "
                                     f"16-byte aligned float32 tensor of {shape}")
                out[name] = t
            else:
                out[name] = torch.empty(shape, dtype=torch.float32, device=dev)
        grads = binding.ImageGrads(d_color.data_ptr() if d_color is not None else None,
                                   d_depth.data_ptr() if d_depth is not None else None,
                                   d_alpha.data_ptr() if d_alpha is not None else None)
        ptr = {k: (v.data_ptr() if v is not None else 0) for k, v in out.items()}
        names = ("means", "log_scales", "quats", "opacity_logits", "sh", "pose")
        if reg is None:
            self.ctx.backward(state, grads, grad_mask, *[ptr[k] for k in names],
                              self.stream_handle())
        else:
            self.ctx.backward_mapping(state, grads, grad_mask, [ptr[k] for k in names], reg,
                                      self.stream_handle())
        return out

    def autotune(self, means, log_scales, quats, opacity_logits, sh, cameras) -> dict:
        """Lets the library pick the fastest tile shape and pixels per thread for this workload
        (cached per scene size and view sizes) and keeps it in this renderer's config."""
        n = int(means.shape[0])
        K = int(sh.shape[1])
        deg = int(round(K ** 0.5)) - 1
        dev = self.device
        t = [_check_param(means, "means", (3,), dev), _check_param(log_scales, "log_scales", (3,), dev),
             _check_param(quats, "quats", (4,), dev),
             _check_param(opacity_logits.reshape(n, 1), "opacity_logits", (1,), dev),
             _check_param(sh, "sh", (K, 3), dev)]
        g = binding.Gaussians(n, deg, *[x.data_ptr() for x in t])
        ms = self.ctx.autotune(g, cameras, self.config, self.stream_handle())
        return dict(tile_w=self.config.tile_w, tile_h=self.config.tile_h,
                    pixels_per_thread=self.config.pixels_per_thread,
                    backward_pixels_per_thread=self.config.backward_pixels_per_thread, ms=ms)

    def release(self, state: int):
        self.ctx.release(state)

    def stats(self, state: int) -> dict:
        return self.ctx.stats(state, self.stream_handle())


class _RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer: Renderer, cameras, means, log_scales, quats, opacity_logits, sh,
                twist):
        cams = binding.make_cameras(cameras)
        color, depth, alpha, state = renderer.forward_raw(means, log_scales, quats,
                                                          opacity_logits, sh, cams)
        ctx.renderer = renderer
        ctx.state = state
        ctx.dims = (int(means.shape[0]), int(sh.shape[1]), len(cams))
        ctx.keep = renderer._last_inputs
        return color, depth, alpha

    @staticmethod
    def backward(ctx, d_color, d_depth, d_alpha):
        needs = ctx.needs_input_grad[2:8]
        mask = 0
        for need, bit in zip(needs, _GRAD_BITS):
            if need:
                mask |= bit
        n, K, V = ctx.dims
        g = {}
        if mask:
            g = ctx.renderer.backward_raw(ctx.state, n, K, V, d_color, d_depth, d_alpha, mask)
        ctx.renderer.release(ctx.state)
        ctx.state = 0
        names = ("means", "log_scales", "quats", "opacity_logits", "sh", "pose")
        return (None, None) + tuple(g.get(k) if need else None for k, need in zip(names, needs))


def render(renderer: Renderer, cameras, means, log_scales, quats, opacity_logits, sh,
           twist: torch.Tensor | None = None):
    """Differentiable render of all `cameras` in one batched launch.

    Returns colour [P,3], depth [P] and accumulated opacity [P] (views concatenated). `twist`
    ([V,6], values ignored: evaluated at zero) receives the per-view pose gradient.
    """
    if twist is None:
        twist = torch.zeros((len(cameras), 6), dtype=torch.float32, device=renderer.device)
    if not torch.is_grad_enabled() or not any(
            t.requires_grad for t in (means, log_scales, quats, opacity_logits, sh, twist)):
        color, depth, alpha, state = renderer.forward_raw(means, log_scales, quats,
                                                          opacity_logits, sh, cameras)
        renderer.release(state)
        return color, depth, alpha
    return _RenderFunction.apply(renderer, cameras, means, log_scales, quats, opacity_logits, sh,
                                 twist)
