"""Pins of the tracking-step oracle (oracle/tracking.py) to things other than itself.

  * exposure fit (Eq. app-ls) == numpy's least-squares solver on the design matrix [C, 1], and
    recovers a planted (g, b) exactly;
  * gradient weights (Eq. app-weight) on images whose central differences are known by hand (a
    ramp, an impulse, a constant, a one-pixel-wide strip) and at the clip;
  * loss and colour gradient (Eq. app-bright, app-trackloss): a hand-computed two-pixel example,
    and the gradient == central finite differences of the loss with (g, b) and the weights held
    at their values;
  * SE(3) exponential == scipy.linalg.expm of the 4x4 twist matrix (the matrix the rasterizer
    oracle's pose gradient is pinned against), over small, moderate and large rotations;
  * Adam: the first step is -lr g / (|g| + eps) by the bias correction, a second step by hand,
    the cosine schedule's end points; the pose moves by exp(xi^) on the left.
  * end to end on the rasterizer oracle: one tracking step from a perturbed pose lowers the
    tracking loss.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import tracking
from paper_2601_00705_gb300 import synthetic


def _cams(*sizes):
    return [dict(width=w, height=h, fx=100.0, fy=100.0, cx=w / 2, cy=h / 2, R=np.eye(3),
                 t=np.zeros(3)) for w, h in sizes]


def _twist(xi):
    M = np.zeros((4, 4))
    M[:3, :3] = [[0.0, -xi[5], xi[4]], [xi[5], 0.0, -xi[3]], [-xi[4], xi[3], 0.0]]
    M[:3, 3] = xi[:3]
    return M


def test_exposure_fit_matches_lstsq_and_recovers_planted_values():
    rng = np.random.default_rng(1)
    cams = _cams((7, 5), (4, 9))
    P = 7 * 5 + 4 * 9
    color = rng.random((P, 3))
    obs = rng.random((P, 3))
    gb = tracking.exposure_fit(color, obs, cams)
    off = 0
    for v, (w, h) in enumerate([(7, 5), (4, 9)]):
        r = color[off:off + w * h].ravel()
        o = obs[off:off + w * h].ravel()
        sol, *_ = np.linalg.lstsq(np.stack([r, np.ones_like(r)], 1), o, rcond=None)
        np.testing.assert_allclose(gb[v], sol, rtol=1e-12, atol=1e-12)
        off += w * h
    planted = 1.3 * color - 0.07
    np.testing.assert_allclose(tracking.exposure_fit(color, planted, cams),
                               [[1.3, -0.07], [1.3, -0.07]], rtol=1e-12, atol=1e-12)


def test_exposure_fit_of_a_constant_render_matches_the_means():
    cams = _cams((3, 2))
    color = np.full((6, 3), 0.25)
    obs = np.arange(18, dtype=float).reshape(6, 3) / 18
    g, b = tracking.exposure_fit(color, obs, cams)[0]
    assert g == 1.0 and b == pytest.approx(obs.mean() - 0.25, abs=1e-15)


def test_grad_weight_on_images_with_known_differences():
    W, H = 6, 4
    cams = _cams((W, H))
    # Horizontal ramp of slope s in every channel: |grad I| = s sqrt(3) everywhere (central
    # differences inside, one-sided on the border, all equal to s on a ramp).
    s, tau = 0.01, 0.05
    ramp = np.repeat((s * np.tile(np.arange(W), H))[:, None], 3, 1)
    np.testing.assert_allclose(tracking.grad_weight(ramp, cams, tau), s * math.sqrt(3) / tau,
                               rtol=1e-12)
    # Constant image: zero; a steep ramp clips at 1.
    np.testing.assert_array_equal(tracking.grad_weight(np.full((W * H, 3), 0.3), cams, tau), 0.0)
    np.testing.assert_array_equal(tracking.grad_weight(10 * ramp, cams, tau), 1.0)
    # Impulse of 1 at (x, y) = (2, 2): its own central differences vanish; the pixel to its left
    # sees (1 - 0) / 2 along x in each channel.
    img = np.zeros((H, W, 3))
    img[2, 2] = 1.0
    w = tracking.grad_weight(img.reshape(-1, 3), cams, 10.0).reshape(H, W)
    assert w[2, 2] == 0.0
    assert w[2, 1] == pytest.approx(0.5 * math.sqrt(3) / 10.0, rel=1e-12)
    assert w[1, 2] == pytest.approx(0.5 * math.sqrt(3) / 10.0, rel=1e-12)
    # Border pixel (x = 0) next to nothing: one-sided difference along y only.
    img = np.zeros((H, W, 3))
    img[1, 0] = 1.0
    w = tracking.grad_weight(img.reshape(-1, 3), cams, 10.0).reshape(H, W)
    assert w[0, 0] == pytest.approx(1.0 * math.sqrt(3) / 10.0, rel=1e-12)  # (I[1]-I[0]) / 1
    # A strip one pixel wide has no x difference.
    cams1 = _cams((1, 5))
    col = np.repeat(np.arange(5.0)[:, None] * 0.01, 3, 1)
    np.testing.assert_allclose(tracking.grad_weight(col, cams1, 1.0), 0.01 * math.sqrt(3),
                               rtol=1e-12)


def test_track_loss_two_pixel_example():
    cams = _cams((2, 1))
    color = np.array([[0.2, 0.4, 0.6], [0.5, 0.5, 0.5]])
    obs = np.array([[0.3, 0.3, 0.9], [0.5, 0.1, 0.7]])
    alpha = np.array([1.0, 0.25])
    wg = np.array([1.0, 0.8])
    loss, d, gb = tracking.track_loss(color, alpha, obs, wg, cams, tau_alpha=0.5,
                                      fit_exposure=False)
    # w = (1, 0.5 * 0.8); residuals (0.1, -0.1, 0.3) and (0, -0.4, 0.2).
    assert loss[0] == pytest.approx(1.0 * 0.5 + 0.4 * 0.6, abs=1e-15)
    np.testing.assert_allclose(d, [[-1.0, 1.0, -1.0], [0.0, 0.4, -0.4]], atol=1e-15)
    np.testing.assert_array_equal(gb, [[1.0, 0.0]])


@pytest.mark.parametrize("fit", [False, True])
def test_track_loss_gradient_matches_finite_differences(fit):
    rng = np.random.default_rng(3 + fit)
    cams = _cams((5, 4), (3, 3))
    P = 29
    color = rng.random((P, 3))
    obs = rng.random((P, 3))
    alpha = rng.random(P)
    wg = rng.random(P)
    loss, d, gb = tracking.track_loss(color, alpha, obs, wg, cams, 0.7, fit_exposure=fit)

    def loss_fixed(c):  # (g, b) and the weights held at their values
        tot = 0.0
        for v, off, n in ((0, 0, 20), (1, 20, 9)):
            g, b = gb[v]
            res = obs[off:off + n] - (g * c[off:off + n] + b)
            w = np.clip(alpha[off:off + n] / 0.7, 0, 1) * wg[off:off + n]
            tot += (w * np.abs(res).sum(-1)).sum()
        return tot

    assert loss.sum() == pytest.approx(loss_fixed(color), rel=1e-12)
    h = 1e-4  # the loss is piecewise linear: exact away from the kinks
    res = obs - (np.repeat(gb, [20, 9], 0)[:, :1] * color + np.repeat(gb, [20, 9], 0)[:, 1:])
    for p in range(P):
        for ch in range(3):
            if abs(res[p, ch]) < 1e-3:
                continue
            cp, cm = color.copy(), color.copy()
            cp[p, ch] += h
            cm[p, ch] -= h
            fd = (loss_fixed(cp) - loss_fixed(cm)) / (2 * h)
            assert d[p, ch] == pytest.approx(fd, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("scale", [1e-7, 1e-3, 0.3, 2.5])
def test_se3_exp_matches_scipy_expm(scale):
    rng = np.random.default_rng(int(scale * 1e7) % 1000)
    for _ in range(5):
        xi = rng.normal(size=6) * scale
        np.testing.assert_allclose(tracking.se3_exp(xi), scipy.linalg.expm(_twist(xi)),
                                   rtol=0, atol=1e-13)
    xi = rng.normal(size=6)
    np.testing.assert_allclose(tracking.se3_exp(xi) @ tracking.se3_exp(-xi), np.eye(4), atol=1e-13)
    rho = np.array([0.1, -0.2, 0.3])
    np.testing.assert_allclose(tracking.se3_exp(np.r_[rho, 0, 0, 0])[:3, 3], rho, atol=1e-16)


def test_adam_first_and_second_step_and_left_update():
    rng = np.random.default_rng(9)
    T = np.stack([np.c_[scipy.linalg.expm(_twist(rng.normal(size=6) * 0.2))[:3, :3],
                        rng.normal(size=3)] for _ in range(2)])
    g1 = rng.normal(size=(2, 6))
    m0 = v0 = np.zeros((2, 6))
    T1, m1, v1, xi1 = tracking.adam_pose_step(T, g1, m0, v0, 0, lr=0.01)
    # Bias correction makes the first step -lr g / (|g| + eps).
    np.testing.assert_allclose(xi1, -0.01 * g1 / (np.abs(g1) + 1e-8), rtol=1e-12)
    for i in range(2):
        Th = np.eye(4)
        Th[:3] = T[i]
        np.testing.assert_allclose(T1[i], (scipy.linalg.expm(_twist(xi1[i])) @ Th)[:3],
                                   atol=1e-13)
    g2 = rng.normal(size=(2, 6))
    _, m2, v2, xi2 = tracking.adam_pose_step(T1, g2, m1, v1, 1, lr=0.01)
    m_hand = 0.9 * 0.1 * g1 + 0.1 * g2
    v_hand = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    np.testing.assert_allclose(m2, m_hand, rtol=1e-14)
    np.testing.assert_allclose(v2, v_hand, rtol=1e-14)
    np.testing.assert_allclose(
        xi2, -0.01 * (m_hand / (1 - 0.9 ** 2)) / (np.sqrt(v_hand / (1 - 0.999 ** 2)) + 1e-8),
        rtol=1e-12)


def test_cosine_schedule_end_points():
    assert tracking.cosine_lr(0, 5e-3, 40) == pytest.approx(5e-3)
    assert tracking.cosine_lr(20, 5e-3, 40) == pytest.approx(2.5e-3)
    assert tracking.cosine_lr(40, 5e-3, 40) == pytest.approx(0.0, abs=1e-18)
    assert tracking.cosine_lr(99, 5e-3, 40) == pytest.approx(0.0, abs=1e-18)
    assert tracking.cosine_lr(7, 5e-3, 0) == 5e-3


def test_one_tracking_step_on_the_rasterizer_oracle_lowers_the_loss():
    wl = synthetic.tiny(seed=11)
    g = wl.gaussians.as_dict()
    cam = dict(wl.cameras[0])
    target = oracle.render(g, [cam])
    obs = target["color"]
    xi_err = np.array([0.02, -0.01, 0.015, 0.01, -0.008, 0.012])
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = cam["R"], cam["t"]
    Tp = scipy.linalg.expm(_twist(xi_err)) @ T
    wgt = tracking.grad_weight(obs, [cam], 0.05)

    def loss_at(Tm):
        c = dict(cam, R=Tm[:3, :3], t=Tm[:3, 3])
        out = oracle.render(g, [c])
        return tracking.track_loss(out["color"], out["alpha"], obs, wgt, [c], 0.5)[0][0], c, out

    l0, c0, out0 = loss_at(Tp)
    _, d_color, _ = tracking.track_loss(out0["color"], out0["alpha"], obs, wgt, [c0], 0.5)
    gpose = oracle.render(g, [c0], d_color=d_color)["g_pose"]
    T1, *_ = tracking.adam_pose_step(Tp[None, :3], gpose, np.zeros((1, 6)), np.zeros((1, 6)), 0,
                                     lr=2e-3)
    T1h = np.eye(4)
    T1h[:3] = T1[0]
    l1 = loss_at(T1h)[0]
    assert l1 < l0


def test_covisibility_hand_counts():
    a = np.array([[0.9, 0.2, 0.6, 0.0, 0.51], [0.0, 0.0, 0.0, 0.0, 0.0]])
    b = np.array([[0.8, 0.7, 0.1, 0.0, 0.5], [0.0, 0.0, 0.0, 0.0, 0.0]])
    inter, union, iou = tracking.covisibility(a, b, 0.5)
    # Pair 0: V_a = {0, 2, 4}, V_b = {0, 1} (0.5 is not above 0.5): intersection {0}, union
    # {0, 1, 2, 4}. Pair 1: both empty.
    assert list(inter) == [1, 0] and list(union) == [4, 0]
    assert list(iou) == [0.25, 0.0]
