"""GPU tests of the tracking step (Eq. app-bright, app-ls, app-trackloss, app-weight; Eq.
leftupdate) against the FP64 oracle in oracle/tracking.py, through the C ABI:
  * a forward with device poses renders bit-identically to one with the same host poses;
  * gradient weights: max-abs 1e-6;
  * exposure fit: relative 1e-5; loss: relative 1e-5; colour gradient: equal (max-abs 1e-6)
    wherever the residual is not within 1e-5 of zero (where FP32 may take the other sign);
  * Adam step and SE(3) update: pose max-abs 1e-6, moments relative 1e-6, step count;
  * one whole iteration against the oracle (render, loss, pose gradient, update): pose max-abs
    2e-5 (the first Adam step is about -lr sign(g), insensitive to the gradient's rounding);
  * a captured iteration replayed from a perturbed pose lowers the loss and the pose error.
"""
import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
from oracle import tracking as otrack
from paper_2601_00705_gb300 import binding, synthetic
from paper_2601_00705_gb300.track import Tracker, poses_of
from gpu_common import renderer, to_dev

pytestmark = pytest.mark.gpu


def _twist(xi):
    M = np.zeros((4, 4))
    M[:3, :3] = [[0.0, -xi[5], xi[4]], [xi[5], 0.0, -xi[3]], [-xi[4], xi[3], 0.0]]
    M[:3, 3] = xi[:3]
    return M


def _perturb(cam, xi):
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = cam["R"], cam["t"]
    Tp = scipy.linalg.expm(_twist(np.asarray(xi, float))) @ T
    # FP32 poses, so that both sides render exactly the same camera.
    return dict(cam, R=Tp[:3, :3].astype(np.float32), t=Tp[:3, 3].astype(np.float32))


def _params(g):
    return [to_dev(g[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]


def _multi_view_scene():
    wl = synthetic.tiny(seed=21)
    base = wl.cameras[0]
    cams = [base,
            dict(synthetic.camera(64, 48, 80.0, 80.0, 31.5, 23.5, np.eye(3), np.zeros(3))),
            _perturb(dict(synthetic.camera(33, 17, 60.0, 60.0, 16.0, 8.0, np.eye(3), np.zeros(3))),
                     [0.05, 0.0, 0.1, 0.02, -0.03, 0.01])]
    return wl.gaussians.as_dict(), cams


def test_posed_forward_is_bit_identical_to_host_poses():
    g, cams = _multi_view_scene()
    r = renderer()
    p = _params(g)
    c0, d0, a0, s0 = r.forward_raw(*p, cams)
    w2c = torch.from_numpy(poses_of(cams)).cuda()
    # The host poses of the cameras are ignored by the posed call: give it wrong ones.
    wrong = [dict(c, R=np.eye(3), t=np.array([5.0, 5.0, 5.0])) for c in cams]
    c1, d1, a1, s1 = r.forward_raw(*p, wrong, world_to_cam=w2c)
    torch.cuda.synchronize()
    for x, y in ((c0, c1), (d0, d1), (a0, a1)):
        assert torch.equal(x, y)
    up = torch.rand_like(c0)
    n, K = int(p[0].shape[0]), int(p[4].shape[1])
    g0 = r.backward_raw(s0, n, K, 3, up, None, None, binding.GRAD_ALL)
    g1 = r.backward_raw(s1, n, K, 3, up, None, None, binding.GRAD_ALL)
    torch.cuda.synchronize()
    for k in g0:
        a, b = g0[k].cpu().numpy(), g1[k].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-12), k
    r.release(s0)
    r.release(s1)


def test_grad_weight_matches_oracle():
    g, cams = _multi_view_scene()
    rng = np.random.default_rng(4)
    P = sum(c["width"] * c["height"] for c in cams)
    obs = oracle.render(g, cams)["color"] + rng.normal(0, 0.01, (P, 3))
    obs = np.clip(obs, 0, 1).astype(np.float32)
    r = renderer()
    w = torch.empty(P, device="cuda")
    obs_d = to_dev(obs)  # held: the kernel reads it after the call returns
    r.ctx.track_grad_weight(binding.make_cameras(cams), obs_d.data_ptr(), 0.05, w.data_ptr(),
                            r.stream_handle())
    torch.cuda.synchronize()
    ref = otrack.grad_weight(obs.astype(np.float64), cams, 0.05)
    np.testing.assert_allclose(w.cpu().numpy(), ref, rtol=0, atol=1e-6)
    assert 0.0 < ref.mean() < 1.0


def _gpu_track_loss(cams, color, alpha, obs, w_grad, tau_alpha, fit):
    r = renderer()
    P, V = color.shape[0], len(cams)
    d = torch.empty((P, 3), device="cuda")
    loss = torch.empty(V, dtype=torch.float64, device="cuda")
    gb = torch.empty((V, 2), device="cuda")
    wg = to_dev(w_grad) if w_grad is not None else None
    cfg = binding.default_track_config(tau_alpha=tau_alpha, fit_exposure=int(fit))
    c_d, a_d, o_d = to_dev(color), to_dev(alpha), to_dev(obs)  # held until the sync below
    r.ctx.track_loss(binding.make_cameras(cams), cfg, c_d.data_ptr(), a_d.data_ptr(),
                     o_d.data_ptr(), wg.data_ptr() if wg is not None else 0, d.data_ptr(),
                     loss.data_ptr(), gb.data_ptr(), r.stream_handle())
    torch.cuda.synchronize()
    return loss.cpu().numpy(), d.cpu().numpy(), gb.cpu().numpy()


@pytest.mark.parametrize("fit,with_w", [(True, True), (False, True), (True, False)])
def test_track_loss_matches_oracle(fit, with_w):
    g, cams = _multi_view_scene()
    rng = np.random.default_rng(5 + fit + 2 * with_w)
    out = oracle.render(g, cams)
    P = out["color"].shape[0]
    color = out["color"].astype(np.float32)
    alpha = out["alpha"].astype(np.float32)
    obs = np.clip(1.15 * out["color"] + 0.03 + rng.normal(0, 0.02, (P, 3)), 0, 1).astype(np.float32)
    w_grad = rng.random(P).astype(np.float32) if with_w else None
    loss, d, gb = _gpu_track_loss(cams, color, alpha, obs, w_grad, 0.5, fit)
    rl, rd, rgb = otrack.track_loss(color.astype(np.float64), alpha.astype(np.float64),
                                    obs.astype(np.float64),
                                    None if w_grad is None else w_grad.astype(np.float64),
                                    cams, 0.5, fit_exposure=fit)
    np.testing.assert_allclose(gb, rgb, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(loss, rl, rtol=1e-5)
    gfull = np.repeat(rgb[:, 0], [c["width"] * c["height"] for c in cams])
    bfull = np.repeat(rgb[:, 1], [c["width"] * c["height"] for c in cams])
    res = obs - (gfull[:, None] * color + bfull[:, None])
    ok = np.abs(res) > 1e-5
    np.testing.assert_allclose(d[ok], rd[ok], rtol=0, atol=1e-6)
    if fit:
        assert np.all(np.abs(rgb[:, 0] - 1.15) < 0.1)


def test_track_loss_planted_exposure_gives_near_zero_loss():
    g, cams = _multi_view_scene()
    out = oracle.render(g, cams)
    color = out["color"].astype(np.float32)
    obs = (0.8 * out["color"] + 0.1).astype(np.float32)
    loss, d, gb = _gpu_track_loss(cams, color, out["alpha"].astype(np.float32), obs, None, 0.5,
                                  True)
    np.testing.assert_allclose(gb, [[0.8, 0.1]] * 3, atol=2e-5)
    assert np.all(loss < 1e-2)


@pytest.mark.parametrize("k,iters", [(0, 0), (3, 0), (5, 20)])
def test_pose_adam_step_matches_oracle(k, iters):
    rng = np.random.default_rng(17 + k)
    V = 5
    T = np.stack([np.c_[scipy.linalg.expm(_twist(rng.normal(size=6) * 0.3))[:3, :3],
                        rng.normal(size=3)] for _ in range(V)]).astype(np.float32)
    grad = (rng.normal(size=(V, 6)) * 10.0 ** rng.integers(-6, 1, size=(V, 6))).astype(np.float32)
    m = (rng.normal(size=(V, 6)) * 0.01 if k else np.zeros((V, 6))).astype(np.float32)
    v = (rng.random(size=(V, 6)) * 0.01 if k else np.zeros((V, 6))).astype(np.float32)
    r = renderer()
    pose = to_dev(T.reshape(V, 12))
    state = to_dev(np.concatenate([m, v], 1))
    step = torch.tensor([k], dtype=torch.int32, device="cuda")
    cfg = binding.default_adam_config(lr=0.01, iterations=iters)
    grad_d = to_dev(grad)  # held until the sync below
    r.ctx.pose_adam_step(V, cfg, grad_d.data_ptr(), state.data_ptr(), step.data_ptr(),
                         pose.data_ptr(), r.stream_handle())
    torch.cuda.synchronize()
    # The C config holds the constants in FP32: the oracle gets the same values.
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    Tn, mn, vn, _ = otrack.adam_pose_step(T.astype(np.float64), grad.astype(np.float64),
                                          m.astype(np.float64), v.astype(np.float64), k,
                                          lr=f32(0.01), beta1=f32(0.9), beta2=f32(0.999),
                                          eps=f32(1e-8), iterations=iters)
    np.testing.assert_allclose(pose.cpu().numpy().reshape(V, 3, 4), Tn, rtol=0, atol=1e-6)
    st = state.cpu().numpy()
    np.testing.assert_allclose(st[:, :6], mn, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(st[:, 6:], vn, rtol=1e-6, atol=1e-18)
    assert int(step.item()) == k + 1


def _tracking_case(seed=11):
    wl = synthetic.tiny(seed=seed)
    g = wl.gaussians.as_dict()
    cam = wl.cameras[0]
    obs = oracle.render(g, [cam])["color"].astype(np.float32)
    start = _perturb(cam, [0.02, -0.01, 0.015, 0.01, -0.008, 0.012])
    return g, cam, start, obs


def test_one_tracking_iteration_matches_oracle():
    g, cam, start, obs = _tracking_case()
    r = renderer()
    p = _params(g)
    tr = Tracker(r, [start], to_dev(obs), lr=2e-3)
    tr.step(*p)
    torch.cuda.synchronize()
    # Oracle: render at the start pose, loss and colour gradient, pose gradient, Adam step.
    wgt = otrack.grad_weight(obs.astype(np.float64), [start], 0.05)
    out = oracle.render(g, [start])
    loss, d_color, gb = otrack.track_loss(out["color"], out["alpha"], obs, wgt, [start], 0.5)
    gpose = oracle.render(g, [start], d_color=d_color)["g_pose"]
    T0 = poses_of([start]).astype(np.float64).reshape(1, 3, 4)
    T1, *_ = otrack.adam_pose_step(T0, gpose, np.zeros((1, 6)), np.zeros((1, 6)), 0, lr=2e-3)
    np.testing.assert_allclose(tr.loss.cpu().numpy(), loss, rtol=1e-3)
    np.testing.assert_allclose(tr.gain_bias.cpu().numpy(), gb, rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(tr.world_to_cam.cpu().numpy().reshape(1, 3, 4), T1, rtol=0,
                               atol=2e-5)
    assert int(tr.step_count.item()) == 1
    r.release(tr.state)


def test_captured_tracking_iterations_lower_loss_and_pose_error():
    g, cam, start, obs = _tracking_case(seed=12)
    r = renderer()
    p = _params(g)
    tr = Tracker(r, [start], to_dev(obs), lr=2e-3, iterations=60)
    tr.step(*p)
    torch.cuda.synchronize()
    first_loss = float(tr.loss.item())
    graph = tr.capture(*p)
    losses = []
    for _ in range(59):
        graph.replay()
        losses.append(float(tr.loss.item()))
    torch.cuda.synchronize()
    assert int(tr.step_count.item()) == 60
    assert losses[-1] < 0.5 * first_loss, (first_loss, losses[::10])
    T_true = poses_of([cam]).reshape(3, 4)
    T_start = poses_of([start]).reshape(3, 4)
    T_end = tr.world_to_cam.cpu().numpy().reshape(3, 4)
    assert np.abs(T_end - T_true).max() < 0.5 * np.abs(T_start - T_true).max()
    r.release(tr.state)


@pytest.mark.parametrize("n,pairs", [(1, 1), (19200, 3), (307200, 2), (0, 2)])
def test_covisibility_matches_oracle(n, pairs):
    rng = np.random.default_rng(n + pairs)
    a = rng.random((pairs, n)).astype(np.float32)
    b = rng.random((pairs, n)).astype(np.float32)
    if n:
        a[0, : n // 3] = 0.0           # some empty and some exactly-at-threshold pixels
        b[-1, : n // 5] = 0.25
    r = renderer()
    ad, bd = to_dev(a), to_dev(b)
    counts = torch.empty((pairs, 2), dtype=torch.int64, device="cuda")
    iou = torch.empty(pairs, device="cuda")
    r.ctx.covisibility(ad.data_ptr(), bd.data_ptr(), n, pairs, 0.25, counts.data_ptr(),
                       iou.data_ptr(), r.stream_handle())
    torch.cuda.synchronize()
    inter, union, ref = otrack.covisibility(a, b, np.float32(0.25))
    np.testing.assert_array_equal(counts.cpu().numpy(), np.stack([inter, union], 1))
    np.testing.assert_array_equal(iou.cpu().numpy(), ref.astype(np.float32))
