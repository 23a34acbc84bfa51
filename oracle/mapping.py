"""FP64 CPU oracle of the mapping regulariser and the maintenance of the Gaussian set (Section
3.5 Eq. reg; appendix "Gaussian Initialization and Joint Mapping": Eq. app-ema, observation
counts, visibility scores, pruning bounds).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module. The product path never imports it, and it imports
nothing from the product package.

Readings where the paper is silent (the CUDA path takes the same ones):
  * Sigma_i^W = R(q_i) diag(exp(2 log_scale_i)) R(q_i)^T; the isotropy term is the Frobenius
    norm of its deviatoric part. Its gradient at an exactly isotropic Gaussian (a kink) is 0.
  * psi(alpha) = -log(alpha) - log(1 - alpha), a barrier against fully transparent and fully
    opaque splats ("avoids degenerate transmittance"), alpha = sigmoid(logit).
  * The anchor mu_bar is held fixed in the gradient.
  * Observation count m_i += the number of views of a forward in which the Gaussian is visible
    (has a touched tile); visibility score v_i += that number times alpha_i.
  * Pruning keeps a Gaussian iff alpha >= min_opacity, tr(Sigma) <= max_trace and not
    (m >= min_observations and v < min_visibility).
  * Non-finite parameters contribute nothing to R.
"""
from __future__ import annotations

import numpy as np


def regularizer(log_scales, logits, means, ema_means, lambda_iso, lambda_alpha, lambda_mu):
    """R of Eq. reg and its gradients. Returns (R, d_log_scales [n,3], d_logits [n],
    d_means [n,3]); ema_means None drops the position term."""
    ls = np.asarray(log_scales, np.float64).reshape(-1, 3)
    lg = np.asarray(logits, np.float64).reshape(-1)
    mu = np.asarray(means, np.float64).reshape(-1, 3)
    n = ls.shape[0]
    d_ls = np.zeros((n, 3))
    d_lg = np.zeros(n)
    d_mu = np.zeros((n, 3))
    total = 0.0
    for i in range(n):
        if not (np.all(np.isfinite(ls[i])) and np.isfinite(lg[i]) and np.all(np.isfinite(mu[i]))):
            continue
        s2 = np.exp(2.0 * ls[i])
        dev = s2 - s2.mean()
        nrm = float(np.sqrt(dev @ dev))
        total += lambda_iso * nrm
        if nrm > 0.0:
            # d nrm / d s2_k = dev_k / nrm (the mean's derivative cancels: sum_k dev_k = 0).
            d_ls[i] += lambda_iso * 2.0 * s2 * dev / nrm
        alpha = 1.0 / (1.0 + np.exp(-lg[i]))
        total += lambda_alpha * (-np.log(alpha) - np.log1p(-alpha))
        d_lg[i] += lambda_alpha * (2.0 * alpha - 1.0)
        if ema_means is not None:
            d = mu[i] - np.asarray(ema_means, np.float64).reshape(-1, 3)[i]
            total += lambda_mu * float(d @ d)
            d_mu[i] += 2.0 * lambda_mu * d
    return total, d_ls, d_lg, d_mu


def ema(means, ema_means, eta):
    """Eq. app-ema: (1 - eta) mu_bar + eta mu."""
    return (1.0 - eta) * np.asarray(ema_means, np.float64) + eta * np.asarray(means, np.float64)


def counters(obs_count, vis_score, views_seen, logits):
    """Maintenance counters after one mapping backward: views_seen[i] = number of views of the
    forward in which Gaussian i is visible."""
    alpha = 1.0 / (1.0 + np.exp(-np.asarray(logits, np.float64)))
    seen = np.asarray(views_seen, np.int64)
    return np.asarray(obs_count, np.int64) + seen, np.asarray(vis_score, np.float64) + seen * alpha


def prune_mask(log_scales, logits, obs_count, vis_score, min_opacity=0.005, max_trace=1.0,
               min_observations=5, min_visibility=1.0):
    alpha = 1.0 / (1.0 + np.exp(-np.asarray(logits, np.float64)))
    tr = np.exp(2.0 * np.asarray(log_scales, np.float64)).sum(-1)
    weak = (np.asarray(obs_count) >= min_observations) & (np.asarray(vis_score) < min_visibility)
    return (alpha >= min_opacity) & (tr <= max_trace) & ~weak
