"""Mapping-side state of the Gaussian set (Section 3.5 Eq. reg; appendix Eq. app-ema and the
maintenance counters used for pruning), on the device through the C ABI.

``MapRegularizer`` owns the EMA anchor, the observation counts and visibility scores of n
Gaussians; ``reg()`` gives the parameter block that ``Renderer.backward_raw(..., reg=...)`` fuses
into the backward (regulariser value and gradients, counter updates); ``update_anchor`` applies
Eq. app-ema after an optimiser step; ``prune_mask`` evaluates the pruning bounds.
"""
from __future__ import annotations

import torch

from . import binding


class MapRegularizer:
    def __init__(self, ctx: binding.Context, means: torch.Tensor, lambda_iso: float = 0.01,
                 lambda_alpha: float = 1e-3, lambda_mu: float = 0.1, eta: float = 0.1):
        dev = means.device
        n = int(means.shape[0])
        self.ctx, self.n, self.eta = ctx, n, float(eta)
        self.lambdas = (float(lambda_iso), float(lambda_alpha), float(lambda_mu))
        self.ema_means = means.detach().to(torch.float32).contiguous().clone()
        self.obs_count = torch.zeros(n, dtype=torch.int32, device=dev)
        self.vis_score = torch.zeros(n, dtype=torch.float32, device=dev)
        self.value = torch.zeros(1, dtype=torch.float64, device=dev)

    def reg(self, anchor: bool = True) -> binding.MapReg:
        li, la, lm = self.lambdas
        return binding.MapReg(li, la, lm, self.ema_means.data_ptr() if anchor else None,
                              self.obs_count.data_ptr(), self.vis_score.data_ptr(),
                              self.value.data_ptr())

    def update_anchor(self, means: torch.Tensor, stream: int = 0):
        """Eq. app-ema after a mapping step: ema = (1 - eta) ema + eta means."""
        m = means.detach().to(torch.float32).contiguous()
        self.ctx.map_ema(self.n, m.data_ptr(), self.ema_means.data_ptr(), self.eta, stream)

    def prune_mask(self, log_scales: torch.Tensor, opacity_logits: torch.Tensor,
                   stream: int = 0, **bounds) -> tuple[torch.Tensor, torch.Tensor]:
        """(keep [n] uint8, number kept [1] int32) by the pruning bounds."""
        ls = log_scales.detach().to(torch.float32).contiguous()
        lg = opacity_logits.detach().to(torch.float32).contiguous()
        keep = torch.empty(self.n, dtype=torch.uint8, device=ls.device)
        n_keep = torch.zeros(1, dtype=torch.int32, device=ls.device)
        self.ctx.prune_mask(self.n, ls.data_ptr(), lg.data_ptr(), self.obs_count.data_ptr(),
                            self.vis_score.data_ptr(), binding.default_prune_config(**bounds),
                            keep.data_ptr(), n_keep.data_ptr(), stream)
        return keep, n_keep
