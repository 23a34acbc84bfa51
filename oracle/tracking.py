"""FP64 CPU oracle of the tracking step around the renderer (Section 3.2 and its appendix: Eq.
app-bright, app-ls, app-trackloss, app-weight; Eq. leftupdate; the Adam optimiser with a cosine
learning-rate schedule) and of the co-visibility measure of keyframe scheduling (Eq. iou).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module. The product path never imports it, and it imports
nothing from the product package.

Plain numpy in float64, written from the equations; no tiling, no fusion. Images are given as
the renderer lays them out: views concatenated, each row-major, colour [P, 3], scalars [P].
Cameras are the same dicts as the rasterizer oracle takes (only width and height are used here).

Readings where the paper is silent (the same readings the CUDA path takes):
  * (g, b) is fitted over all pixels and the three channels of a view, without weights
    (Eq. app-ls); a render with no variance gets g = 1 and b = mean(I) - mean(rendered).
  * (g, b) and the weights are held fixed in the gradient: they are re-estimated from every
    render, and no gradient flows into them.
  * grad I is the central difference per channel inside the image, one-sided on its border and
    zero along an axis of extent 1; ||grad I||_2 is taken over both axes and the three channels.
  * The loss is the plain sum of Eq. app-trackloss (no normalisation) with sign(0) = 0.
  * Adam with bias correction (beta1 0.9, beta2 0.999, eps 1e-8); the learning rate of step k is
    lr (1 + cos(pi min(k, K) / K)) / 2 for a schedule of K steps, or lr when K = 0.
  * The twist xi = (rho, omega) acts on the left: T <- exp(xi^) T, with the SE(3) exponential
    of the 4x4 matrix [[omega]_x, rho; 0, 0].
  * Co-visibility (Eq. iou): the main text counts visible Gaussians, the appendix visible
    pixels; the pixel form is used, V = {p : accumulated opacity > tau}, compared pixel by
    pixel between the two frames, and IoU = 0 when both masks are empty.
"""
from __future__ import annotations

import math

import numpy as np


def _views(cameras):
    """(pixel offset, width, height) of each view."""
    out, off = [], 0
    for c in cameras:
        w, h = int(c["width"]), int(c["height"])
        out.append((off, w, h))
        off += w * h
    return out


def grad_weight(observed, cameras, tau_grad):
    """w(p) = clip(||grad I(p)||_2 / tau_grad, 0, 1) per pixel (Eq. app-weight)."""
    obs = np.asarray(observed, dtype=np.float64).reshape(-1, 3)
    w = np.zeros(obs.shape[0])
    for off, W, H in _views(cameras):
        img = obs[off:off + W * H].reshape(H, W, 3)
        gx = np.zeros_like(img)
        gy = np.zeros_like(img)
        for x in range(W):
            xl, xr = max(x - 1, 0), min(x + 1, W - 1)
            if xr > xl:
                gx[:, x] = (img[:, xr] - img[:, xl]) / (xr - xl)
        for y in range(H):
            yu, yd = max(y - 1, 0), min(y + 1, H - 1)
            if yd > yu:
                gy[y] = (img[yd] - img[yu]) / (yd - yu)
        norm = np.sqrt((gx ** 2).sum(-1) + (gy ** 2).sum(-1))
        w[off:off + W * H] = np.clip(norm / tau_grad, 0.0, 1.0).ravel()
    return w


def exposure_fit(color, observed, cameras):
    """(g, b) per view minimising sum ||I - g C - b||^2 over pixels and channels (Eq. app-ls),
    from the normal equations of the two-parameter least-squares problem."""
    col = np.asarray(color, dtype=np.float64).reshape(-1, 3)
    obs = np.asarray(observed, dtype=np.float64).reshape(-1, 3)
    gb = np.zeros((len(cameras), 2))
    for v, (off, W, H) in enumerate(_views(cameras)):
        r = col[off:off + W * H].ravel()
        o = obs[off:off + W * H].ravel()
        n = r.size
        sr, srr, so, sro = r.sum(), (r * r).sum(), o.sum(), (r * o).sum()
        den = n * srr - sr * sr
        if n > 0 and den > 1e-12 * n * n:
            g = (n * sro - sr * so) / den
            b = (so - g * sr) / n
        else:
            g = 1.0
            b = (so - sr) / n if n else 0.0
        gb[v] = (g, b)
    return gb


def track_loss(color, alpha, observed, w_grad, cameras, tau_alpha, fit_exposure=True):
    """Weighted L1 loss per view with the affine brightness model and its gradient with respect
    to the rendered colour (Eq. app-bright, app-trackloss, app-weight).

    Returns (loss [V], d_color [P, 3], gain_bias [V, 2])."""
    col = np.asarray(color, dtype=np.float64).reshape(-1, 3)
    a = np.asarray(alpha, dtype=np.float64).reshape(-1)
    obs = np.asarray(observed, dtype=np.float64).reshape(-1, 3)
    wg = np.ones(a.shape[0]) if w_grad is None else np.asarray(w_grad, dtype=np.float64).reshape(-1)
    gb = exposure_fit(col, obs, cameras) if fit_exposure else np.tile([1.0, 0.0], (len(cameras), 1))
    loss = np.zeros(len(cameras))
    d_color = np.zeros_like(col)
    for v, (off, W, H) in enumerate(_views(cameras)):
        sl = slice(off, off + W * H)
        g, b = gb[v]
        res = obs[sl] - (g * col[sl] + b)
        w = np.clip(a[sl] / tau_alpha, 0.0, 1.0) * wg[sl]
        loss[v] = (w * np.abs(res).sum(-1)).sum()
        d_color[sl] = -(w * g)[:, None] * np.sign(res)
    return loss, d_color, gb


def skew(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def se3_exp(xi):
    """4x4 SE(3) exponential of xi = (rho, omega) (closed form: Rodrigues for the rotation and
    the left Jacobian V for the translation; series below |omega|^2 = 1e-10)."""
    xi = np.asarray(xi, dtype=np.float64)
    rho, om = xi[:3], xi[3:]
    th2 = float(om @ om)
    if th2 < 1e-10:
        A, B, C = 1.0 - th2 / 6.0, 0.5 - th2 / 24.0, 1.0 / 6.0 - th2 / 120.0
    else:
        th = math.sqrt(th2)
        A, B, C = math.sin(th) / th, (1.0 - math.cos(th)) / th2, (th - math.sin(th)) / (th2 * th)
    W = skew(om)
    R = np.eye(3) + A * W + B * (W @ W)
    V = np.eye(3) + B * W + C * (W @ W)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ rho
    return T


def cosine_lr(k, lr, iterations):
    if iterations <= 0:
        return lr
    return 0.5 * lr * (1.0 + math.cos(math.pi * min(k, iterations) / iterations))


def adam_pose_step(world_to_cam, d_pose, m, v, k, lr=5e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   iterations=0):
    """One Adam step on the twist of every view, applied on the left (Eq. leftupdate).

    world_to_cam [V, 3, 4]; d_pose [V, 6] = dL/dxi at xi = 0; m, v [V, 6]; k = steps taken.
    Returns (new world_to_cam, m, v, xi [V, 6])."""
    T0 = np.asarray(world_to_cam, dtype=np.float64).reshape(-1, 3, 4)
    g = np.asarray(d_pose, dtype=np.float64).reshape(-1, 6)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** (k + 1))
    vhat = v / (1.0 - beta2 ** (k + 1))
    xi = -cosine_lr(k, lr, iterations) * mhat / (np.sqrt(vhat) + eps)
    out = np.empty_like(T0)
    for i in range(T0.shape[0]):
        T = np.eye(4)
        T[:3] = T0[i]
        out[i] = (se3_exp(xi[i]) @ T)[:3]
    return out, m, v, xi


def covisibility(alpha_a, alpha_b, tau):
    """Eq. iou with the per-pixel visibility masks: V = {p : alpha(p) > tau} for each image of a
    pair; returns (intersection, union, IoU), IoU = 0 for an empty union. alpha_* [n_pairs, n]."""
    va = np.asarray(alpha_a, dtype=np.float64) > tau
    vb = np.asarray(alpha_b, dtype=np.float64) > tau
    inter = (va & vb).sum(-1)
    union = (va | vb).sum(-1)
    iou = np.where(union > 0, inter / np.maximum(union, 1), 0.0)
    return inter, union, iou
