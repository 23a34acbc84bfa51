"""Pose tracking on the device: the tracking step around the renderer (Section 3.2 and its
appendix: Eq. app-bright, app-ls, app-trackloss, app-weight; Eq. leftupdate).

One iteration renders every view at its current device pose, fits the exposure (g, b) per view,
forms the weighted L1 loss and its colour gradient, back-propagates to the pose twists only and
takes one Adam step T <- exp(xi^) T per view. Nothing in an iteration synchronises with the host,
so a whole iteration can be captured once and replayed (``Tracker.capture``).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding
from .render import Renderer


def poses_of(cameras) -> np.ndarray:
    """Row-major [R|t] of each camera dict, as float32 [V,12]."""
    out = np.zeros((len(cameras), 12), dtype=np.float32)
    for v, c in enumerate(cameras):
        out[v] = np.concatenate([np.asarray(c["R"], np.float64).reshape(3, 3),
                                 np.asarray(c["t"], np.float64).reshape(3, 1)], 1).ravel()
    return out


class Tracker:
    """Tracks the poses of V views against observed frames with the map held fixed.

    observed: device float32 [P,3] frames (views concatenated as the renderer lays them out).
    world_to_cam: initial poses, float32 [V,12] (host or device); default: the cameras' poses.
    Loss constants: tau_alpha, tau_grad, fit_exposure; Adam: lr, betas, eps, iterations (cosine
    schedule length, 0 = constant lr).
    """

    def __init__(self, renderer: Renderer, cameras, observed: torch.Tensor,
                 world_to_cam=None, *, tau_alpha: float = 0.5, tau_grad: float = 0.05,
                 fit_exposure: bool = True, lr: float = 5e-3, betas=(0.9, 0.999),
                 eps: float = 1e-8, iterations: int = 0):
        self.r = renderer
        dev = renderer.device
        self.cameras = list(cameras)
        self.cams = binding.make_cameras(self.cameras)
        V = len(self.cams)
        P = sum(int(c.width) * int(c.height) for c in self.cams)
        if observed.shape != (P, 3) or observed.dtype != torch.float32 or observed.device != dev:
            raise ValueError(f"observed must be a float32 [{P},3] tensor on {dev}")
        self.observed = observed.contiguous()
        init = poses_of(self.cameras) if world_to_cam is None else world_to_cam
        self.world_to_cam = torch.as_tensor(init, dtype=torch.float32).reshape(V, 12).to(dev).clone()
        self.track_cfg = binding.default_track_config(tau_alpha=float(tau_alpha),
                                                      tau_grad=float(tau_grad),
                                                      fit_exposure=int(bool(fit_exposure)))
        self.adam_cfg = binding.default_adam_config(lr=float(lr), beta1=float(betas[0]),
                                                    beta2=float(betas[1]), eps=float(eps),
                                                    iterations=int(iterations))
        self.adam_state = torch.zeros((V, 12), dtype=torch.float32, device=dev)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.w_grad = torch.empty(P, dtype=torch.float32, device=dev)
        renderer.ctx.track_grad_weight(self.cams, self.observed.data_ptr(), float(tau_grad),
                                       self.w_grad.data_ptr(), renderer.stream_handle())
        self.images = (torch.empty((P, 3), device=dev), torch.empty(P, device=dev),
                       torch.empty(P, device=dev))
        self.d_color = torch.empty((P, 3), dtype=torch.float32, device=dev)
        self.loss = torch.zeros(V, dtype=torch.float64, device=dev)
        self.gain_bias = torch.zeros((V, 2), dtype=torch.float32, device=dev)
        self.d_pose = torch.zeros((V, 6), dtype=torch.float32, device=dev)
        self.state = 0

    def step(self, means, log_scales, quats, opacity_logits, sh) -> None:
        """One tracking iteration on the current stream (asynchronous). The loss of the poses
        this iteration started from is left in ``self.loss``."""
        r = self.r
        stream = r.stream_handle()
        color, _, alpha, self.state = r.forward_raw(means, log_scales, quats, opacity_logits, sh,
                                                    self.cams, state=self.state, out=self.images,
                                                    world_to_cam=self.world_to_cam)
        r.ctx.track_loss(self.cams, self.track_cfg, color.data_ptr(), alpha.data_ptr(),
                         self.observed.data_ptr(), self.w_grad.data_ptr(), self.d_color.data_ptr(),
                         self.loss.data_ptr(), self.gain_bias.data_ptr(), stream)
        n, K = int(means.shape[0]), int(sh.shape[1])
        r.backward_raw(self.state, n, K, len(self.cams), self.d_color, None, None,
                       binding.GRAD_POSE, out={"pose": self.d_pose})
        r.ctx.pose_adam_step(len(self.cams), self.adam_cfg, self.d_pose.data_ptr(),
                             self.adam_state.data_ptr(), self.step_count.data_ptr(),
                             self.world_to_cam.data_ptr(), stream)

    def capture(self, means, log_scales, quats, opacity_logits, sh) -> torch.cuda.CUDAGraph:
        """Captures one iteration as a CUDA graph (after an eager iteration has sized the
        renderer's buffers: call ``step`` once first). Each replay is one more iteration."""
        dev = self.r.device
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.step(means, log_scales, quats, opacity_logits, sh)
        torch.cuda.current_stream(dev).wait_stream(s)
        return g
